/*
 * pycool.h -- C ABI of the GB300-native symplectic lattice stepper.
 *
 * The library evolves N_f real scalar fields phi_i and their momenta pi_i on a
 * periodic n^3 lattice in a flat FRW background (scale factor a, momentum
 * p_a), with the split-Hamiltonian symplectic integrators of J. Sainio,
 * "PyCOOL" (arXiv:1201.5029):
 *   - the three exact sub-flows Phi_H1, Phi_H2, Phi_H3 (Sec. 2.3, Eq. split-Phi),
 *   - composed into the second-order stage
 *       Phi1(h/2) Phi2(h/2) Phi3(h) Phi2(h/2) Phi1(h/2)   (Sec. 2.3, after Eq. split-Phi),
 *   - composed into orders 4 (triple jump, Eq. Phi-rec), 6 and 8 (Table 1).
 * Time is conformal time; dt is the conformal step d-eta.
 *
 * Conventions shared by every call:
 *   - Field arrays are float64, layout [field][z][y][x] (x fastest), n^3 sites
 *     per field, N_f fields (1 or 2, fixed by the model).
 *   - Every call returns a pycool_status and never aborts.  Asynchronous errors
 *     (a CUDA fault, a non-finite lattice sum) are latched in the simulation and
 *     returned by the next pycool_sync / pycool_energies / pycool_get_fields.
 *     After PYCOOL_E_CUDA the simulation answers PYCOOL_E_STATE until destroyed.
 *   - A simulation is used by one host thread at a time.  Server calls are
 *     thread-safe.
 *   - All device work of a simulation is ordered on the CUDA stream given at
 *     creation; no call other than pycool_sync/energies/get_fields(host)/
 *     field_stats blocks the host.
 */
#ifndef PYCOOL_H
#define PYCOOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PYCOOL_MAX_FIELDS 2
#define PYCOOL_MAX_PARAMS 8

typedef struct pycool_sim pycool_sim;
typedef struct pycool_server pycool_server;

typedef enum {
  PYCOOL_OK = 0,
  PYCOOL_E_INVALID = 1,      /* bad argument or configuration                      */
  PYCOOL_E_UNSTABLE_DT = 2,  /* dt breaks the linear stability bound at a = 1     */
  PYCOOL_E_NOMEM = 3,        /* device or host allocation failed / budget exceeded */
  PYCOOL_E_CUDA = 4,         /* a CUDA call failed; the simulation is poisoned    */
  PYCOOL_E_NONFINITE = 5,    /* a lattice sum became NaN or Inf                   */
  PYCOOL_E_TIMEOUT = 6,      /* a wait ran past its deadline                      */
  PYCOOL_E_STATE = 7,        /* call not valid in the current state               */
  PYCOOL_E_BUSY = 8,         /* server queue full                                 */
  PYCOOL_E_NOT_FOUND = 9,    /* unknown ticket                                    */
  PYCOOL_E_CANCELLED = 10    /* the request was cancelled before it finished      */
} pycool_status;

/* Potentials (Sec. 3).  params[] per model:
 *   FREE     : V = m2/2 phi^2                                      {m2}
 *   CHAOTIC2 : V = m2/2 phi^2 + g2/2 phi^2 chi^2   (Sec. 3.1)      {m2, g2}
 *   OSCILLON : V = m2/2 phi^2 - lam/4 phi^4 + g/6 phi^6 (Sec. 3.2) {m2, lam, g}
 *   QBALL    : V = m2 |Phi|^2 (1 + K ln(|Phi|^2/M^2)),
 *              |Phi|^2 = (phi_1^2 + phi_2^2)/2          (Sec. 3.3) {m2, K, M}
 * FREE and OSCILLON have one field; CHAOTIC2 and QBALL have two. */
typedef enum {
  PYCOOL_MODEL_FREE = 0,
  PYCOOL_MODEL_CHAOTIC2 = 1,
  PYCOOL_MODEL_OSCILLON = 2,
  PYCOOL_MODEL_QBALL = 3
} pycool_model;

/* Arithmetic of the bulk sweep.
 *   FP64       : fields, momenta and all arithmetic in float64.
 *   SPLIT_FP32 : phi_i = phi0_i + dphi_i, pi_i = pi0_i + dpi_i with the lattice
 *                means phi0, pi0 in float64 and the fluctuations dphi, dpi
 *                stored and updated in float32; lattice sums, a and p_a in
 *                float64 (the homogeneous/perturbation split of Sec. 2.2,
 *                Eq. phi-lin, used here for precision, not linearisation).
 *   SPLIT_DD   : the same split with the fluctuations stored and updated as
 *                double-float pairs (hi + lo float32, ~48-bit significand,
 *                8 bytes per value like FP64): float64-class accuracy with the
 *                bulk arithmetic on the FP32 pipe (error-free transformations
 *                TwoSum and the FMA-based TwoProduct).  Needs n a multiple of
 *                32 (the persistent kernel); the server does not take it. */
typedef enum { PYCOOL_FP64 = 0, PYCOOL_SPLIT_FP32 = 1, PYCOOL_SPLIT_DD = 2 } pycool_precision;

/* Discrete Laplacian D of Sec. 2.1, Eq. D (its coefficients are not printed):
 *   7PT   : c = (-6, 1, 0, 0) for (centre, face, edge, corner) neighbours,
 *   ISO27 : c = (-128, 14, 3, 1)/30 (isotropic at O(k^4)),
 *   4TH   : the fourth-order stencil Sec. 2.1 mentions (HLATTICE's, not
 *           printed): per axis (-1, 16, -30, 16, -1)/12 over two sites each
 *           way, 13 points; symbol -k^2 + O(k^6).  n >= 4.  FP64: the
 *           persistent kernel when n % 32 == 0, else a per-stage kernel;
 *           SPLIT_DD: the persistent kernel, n % 32 == 0 (E_INVALID otherwise);
 *           SPLIT_FP32: the per-stage kernel.  No linearised path. */
typedef enum {
  PYCOOL_STENCIL_7PT = 7,
  PYCOOL_STENCIL_4TH = 13,
  PYCOOL_STENCIL_ISO27 = 27
} pycool_stencil;

/* Time step rule.
 *   CONFORMAL : every time step advances conformal time by dt (d-eta = dt).
 *   PHYSICAL  : the adaptive conformal step of Sec. 3.1 -- each time step
 *               advances physical time (dt_phys = a d-eta) by about dt:
 *               d-eta = dt / a_n, a_n the scale factor of the synchronised
 *               state that starts the step; all stages of the step use it. */
typedef enum { PYCOOL_TIME_CONFORMAL = 0, PYCOOL_TIME_PHYSICAL = 1 } pycool_time_step;

typedef struct {
  int32_t n;          /* lattice side, 1 <= n <= 1024; S = V_L = n^3 (Sec. 2.1)       */
  int32_t model;      /* pycool_model                                                */
  int32_t order;      /* integrator order: 2, 4, 6 or 8                              */
  int32_t precision;  /* pycool_precision                                            */
  int32_t stencil;    /* pycool_stencil                                              */
  int32_t time_step;  /* pycool_time_step (0 = conformal)                            */
  double L;           /* comoving box side; dx = L/n                                 */
  double dt;          /* time step (conformal d-eta, or physical dt: time_step);     */
                      /* may be negative (time reversal)                             */
  double mpl;         /* reduced Planck mass in program units; +INF = static a       */
  double rho_rad0;    /* homogeneous radiation density today-units (Eq. H2)          */
  double rho_mat0;    /* homogeneous matter density (Eq. H2)                         */
  double params[PYCOOL_MAX_PARAMS]; /* model parameters, see pycool_model            */
} pycool_config;

/* Observables at a synchronised state (all fields at the same time eta).
 * rho_kin[i]  = sum pi_i^2 / (2 a^6 S)
 * rho_grad[i] = -sum phi_i D[phi_i] / (2 a^2 dx^2 S)     (Stokes identity, Sec. 2.1)
 * rho_pot     = sum V / S
 * rho         = sum_i (rho_kin[i] + rho_grad[i]) + rho_pot         (Eq. rho-pres)
 * P           = sum_i (rho_kin[i] - rho_grad[i]/3) - rho_pot       (Eq. rho-pres)
 * H           = a'/a^2 = -p_a / (6 S m_pl^2 a^2)                    (Eq. a)
 * residual    = |(rho + rho_rad0/a^4 + rho_mat0/a^3) / (3 m_pl^2 H^2) - 1|  (Eq. res-curv)
 * mean[i], variance[i]: lattice mean and variance of phi_i. */
typedef struct {
  double eta, a, pa, H;
  double rho_kin[PYCOOL_MAX_FIELDS];
  double rho_grad[PYCOOL_MAX_FIELDS];
  double rho_pot, rho, P, residual;
  double mean[PYCOOL_MAX_FIELDS];
  double variance[PYCOOL_MAX_FIELDS];
  int64_t steps_done;   /* completed time steps since set_initial */
  int64_t sweeps_done;  /* fused stage sweeps launched (one per Phi^(2) stage) */
} pycool_observables;

/* ---- single simulation ------------------------------------------------------ */

/* Number of Phi^(2) stages per time step for an order (1, 3, 7, 15), or -1. */
int pycool_stages_per_step(int32_t order);

/* Stage weights w_1..w_s of one step in the order applied (Eq. Phi-rec for
 * order 4, Table 1 for orders 6 and 8).  w must hold 15 doubles. */
pycool_status pycool_stage_weights(int32_t order, double* w, int32_t* count);

/* Bytes of device memory a simulation needs: state_bytes holds the field
 * buffers and the background record, workspace_bytes the per-block partial
 * sums of the reductions.  Returns E_INVALID for a bad config. */
pycool_status pycool_query_bytes(const pycool_config* cfg, size_t* state_bytes,
                                 size_t* workspace_bytes);

/* Create a simulation of the problem of Sec. 3 ("model file": lattice n, box L,
 * dt, potential, integrator order).
 *   dev_state / dev_workspace : device buffers of at least the queried sizes,
 *       256-byte aligned, owned by the caller and valid until pycool_destroy;
 *       NULL = the library allocates (and frees) its own.
 *   cuda_stream : cudaStream_t the simulation's work is ordered on (NULL = the
 *       legacy default stream).  Not retained beyond the simulation's life.
 * Checks the linear stability bound |h| omega_max < 2 at a = 1 for every stage
 * weight (omega_max^2 = max|symbol of D|/dx^2 + m2) -> E_UNSTABLE_DT.
 * The device must be current on the calling thread. */
pycool_status pycool_create(const pycool_config* cfg, void* dev_state, void* dev_workspace,
                            void* cuda_stream, pycool_sim** out);

/* Initial fields and momenta, float64 [field][z][y][x], N_f n^3 values each.
 * on_device != 0: phi and pi are device pointers (read on the stream).
 * on_device == 0: host pointers, copied before the call returns.
 * a0 > 0 is the initial scale factor.  pa0 = NaN: p_a is the negative root of
 * the Hamiltonian constraint H = 0 (Eq. H2; expanding branch, p_a < 0, Eq. p-a);
 * for mpl = +INF, p_a = 0.  For the split forms the lattice mean of each field
 * and momentum (a compensated sum in a fixed order on the device) is taken as
 * the float64 background and the rest, x - mean, is rounded to float32
 * (SPLIT_FP32) or split into a double-float pair hi + lo (SPLIT_DD), all in
 * kernels; host inputs are staged in the simulation's own field buffers, so
 * the call allocates nothing. */
pycool_status pycool_set_initial(pycool_sim* sim, const double* phi, const double* pi,
                                 int on_device, double a0, double pa0);

/* Advance by `steps` time steps of the chosen order (one fused sweep per
 * Phi^(2) stage, then one drift-only sweep that synchronises phi with pi).
 * Asynchronous: returns once the work is queued on the stream. */
pycool_status pycool_evolve(pycool_sim* sim, int64_t steps);

/* Wait until the simulation's queued work is done, at most timeout_s seconds
 * (<0: no limit).  Returns a latched error if any, else E_TIMEOUT or OK. */
pycool_status pycool_sync(pycool_sim* sim, double timeout_s);

/* Synchronise, then fill *out with the observables of the current state. */
pycool_status pycool_energies(pycool_sim* sim, pycool_observables* out);

/* Mean and variance of field `field` at the current state (synchronises). */
pycool_status pycool_field_stats(pycool_sim* sim, int32_t field, double* mean,
                                 double* variance);

/* Copy the current fields and momenta out, float64 [field][z][y][x]
 * (split forms: phi0 + dphi evaluated in float64 by a kernel; host outputs go
 * through the field buffer the current state does not use).  on_device as for
 * set_initial; the call synchronises.  Either pointer may be NULL. */
pycool_status pycool_get_fields(pycool_sim* sim, double* phi, double* pi, int on_device);

/* ---- potentials given at run time --------------------------------------------
 * The analogue of the paper's model files (Sec. 2.4: the potential strings of
 * a model are turned into CUDA code at run time): the caller gives V and
 * dV/dphi_i as C expressions in the fields f0 (and f1) and the parameters
 * p[0..7] (the config's params), e.g. "0.5*p[0]*f0*f0 + 0.25*p[1]*f0*f0*f0*f0";
 * the library compiles them with NVRTC into one kernel for this device and
 * returns a model id (>= 16) to put in pycool_config.model.  Such a model
 * runs in the FP64 form with any of the three stencils, one stage as
 * three launches (the library's drift, the compiled potential, the library's
 * stencil, kick and sums); params[0] is taken as the mass scale m^2 of the
 * stability check.  pycool_energy_fields runs the compiled kernel on the
 * current fields for V.  Not available with such models: the split forms,
 * the server, the allocation-free sweep and the linearised evolution
 * (E_INVALID).  The expressions are compiled into the
 * caller's own process; a compile error returns E_INVALID and prints the
 * compiler's log to stderr.  E_CUDA: the compiled kernel could not be
 * loaded (no GPU); E_NOMEM: 64 models already defined in this process.
 * pycool_model_source gives the generated kernel source (len: its length
 * without the terminating zero; buf may be NULL). */
pycool_status pycool_model_define(int32_t nf, const char* V, const char* const* dV,
                                  int32_t* model_id);
pycool_status pycool_model_source(int32_t model_id, char* buf, size_t cap, size_t* len);

/* ---- output-interval observables (computed on the device) ------------------
 * pycool_energy_fields: the energy density and pressure at every site of the
 *   current synchronised state (synchronises first), Sec. 2.1 Eq. rho-pres
 *   with the gradient terms from the stencil G of Eq. G and phi' = pi/a^2:
 *     rho = sum_i [pi_i^2/(2 a^6) + G[phi_i]/(2 a^2 dx^2)] + V(phi)
 *     P   = sum_i [pi_i^2/(2 a^6) - G[phi_i]/(6 a^2 dx^2)] - V(phi)
 *     G[phi](x) = 1/2 sum_alpha c_d(alpha) (phi(alpha) - phi(x))^2
 *   (c_d of the configured stencil).  Their lattice means are the rho and P
 *   of pycool_energies (Stokes identity).  rho, P: n^3 float64 [z][y][x],
 *   device pointers if on_device, else host (the call then allocates two
 *   device arrays for the duration).
 * pycool_spectrum_bins: number of shells of an n^3 lattice's spectrum,
 *   floor(sqrt(3) n / 2) + 2 (-1 for a bad n).
 * pycool_spectrum: the power spectrum of field `field` (which = 0) or of its
 *   momentum (which = 1) at the current synchronised state (Sec. 2.4's field
 *   spectra; the paper does not define them: this library's definition):
 *     power[b] = sum over modes k with round(|m_k|) = b of |F_k|^2 / S^2,
 *     count[b] = number of those modes (may be NULL),
 *   F the unnormalised forward transform of the field, m_k the signed integer
 *   wave vector; the shells add up to the lattice mean of the field squared.
 *   power, count: host arrays of nbins = pycool_spectrum_bins(n).  The first
 *   call makes an FFT plan and device buffers that the simulation keeps.
 * Errors: E_INVALID (bad arguments), E_STATE (no synchronised state), E_NOMEM,
 * E_CUDA, and the latched errors of pycool_sync. */
pycool_status pycool_energy_fields(pycool_sim* sim, double* rho, double* P, int on_device);
int32_t pycool_spectrum_bins(int32_t n);
pycool_status pycool_spectrum(pycool_sim* sim, int32_t which, int32_t field, double* power,
                              int64_t* count, int32_t nbins);

/* Checkpoint of a synchronised state: the background record (eta, a, p_a,
 * step counters, split background phi0/pi0) and the current fields and
 * momenta in the sweep's own precision.  pycool_checkpoint_size gives the
 * byte count; save copies into a host buffer of at least that size
 * (synchronises; E_STATE if work is pending); load restores it into a
 * simulation created with the same config, so that evolving on continues bit
 * for bit as the saved simulation would have. */
pycool_status pycool_checkpoint_size(pycool_sim* sim, size_t* size);
pycool_status pycool_checkpoint_save(pycool_sim* sim, void* buf, size_t cap);
pycool_status pycool_checkpoint_load(pycool_sim* sim, const void* buf, size_t size);

/* Replace the stream the simulation's work is ordered on (synchronises first). */
pycool_status pycool_set_stream(pycool_sim* sim, void* cuda_stream);

/* Number of this library's kernels the simulation has launched so far
 * (sweeps, arming and conversion kernels), for accounting; -1 for NULL. */
int64_t pycool_kernel_launches(const pycool_sim* sim);

/* Work plan of the persistent evolve kernel that pycool_evolve uses for n a
 * multiple of 32 (host arithmetic only: no device call, no GPU needed).  The
 * lattice is cut into tiles of (32 vx) x 16 sites (vx = sites per thread in
 * x), each tile's z-axis into ranges, and the (tile, z-range) units are dealt
 * to at most `sms` blocks so that the blocks' modelled work is even; the
 * model depends on whether a stage's traffic fits the device's L2 of
 * l2_bytes (pycool_evolve passes the device's SM count and L2 size).
 *   stencil: a pycool_stencil; 4TH (the FP64 and SPLIT_DD forms only) loads
 *       two halo planes, rows and columns per side, the others one
 *   geo (out, 10 int32): n, vx, tile width, tiles in x, tiles, z-chunks per
 *       tile clear of the periodic y boundary, per tile at it, units, blocks G,
 *       z-halo planes per side H
 *   units (out, 4 int32 per unit, room for cap_units units, may be NULL):
 *       x0, y0, z0, planes + 2 H (the planes loaded: the range and its z halo),
 *       block by block, each block's in processing order
 *   uoff (out, room for cap_blocks + 1, may be NULL): block b's units are
 *       units[uoff[b] .. uoff[b + 1])
 * Every (tile, z) pair of the lattice belongs to exactly one unit.
 * E_INVALID: n not a positive multiple of 32, nf not 1 or 2, precision not a
 * pycool_precision, stencil not a pycool_stencil or 4TH with SPLIT_FP32,
 * sms < 1, l2_bytes < 0, or arrays too small for the plan. */
pycool_status pycool_persist_plan(int32_t n, int32_t nf, int32_t precision, int32_t stencil,
                                  int32_t sms, int64_t l2_bytes, int32_t* geo, int32_t* units,
                                  int32_t cap_units, int32_t* uoff, int32_t cap_blocks);

/* Growth functions of the linearised evolution (Sec. 2.2, Eqs. a-lin, phi-0,
 * Phik-1): the homogeneous background (a, p_a, phi0, pi0) evolved without the
 * perturbations, and for each of nk values of k_eff^2 (the symbol of the
 * discrete Laplacian, dimensionless: -D applied to a plane wave) the
 * 2N_f x 2N_f matrix T with (dPhi_k, dPi_k)(eta) = T (dPhi_k, dPi_k)(0) for
 * every Fourier mode k of the perturbations with that k_eff^2, after `steps`
 * time steps of the configuration's order, time-step rule (dt, or the
 * physical-time step dt / a at each step's start) and potential (n and L set
 * V_L and dx; precision and stencil are not used).  The equations of the modes
 * are linear, so modes with equal k_eff^2 share one T: the caller reconstructs
 * each mode as T times its initial values.
 *   phi0, pi0 (in, N_f each): the initial background fields and momenta;
 *     a0 > 0, pa0: scale factor and its momentum
 *   k2 (in, host, nk values); T (out, host, nk x (2N_f)^2 doubles, row-major
 *     per value, rows dPhi_1..dPhi_N, dPi_1..dPi_N, columns the initial
 *     components in the same order); background (out, host, 2 + 2 N_f doubles:
 *     a, p_a, phi0[N_f], pi0[N_f] at the end)
 * Work on `cuda_stream` (NULL: the default stream); the call allocates its
 * device buffers and synchronises the stream before it returns.
 * Errors: E_INVALID (bad config or arguments), E_UNSTABLE_DT, E_NOMEM, E_CUDA.
 * The Q-ball's second derivatives need |Phi0| > 0 throughout. */
/* The distinct k_eff^2 values of an n^3 lattice (host arithmetic only): the
 * symbol of -D (Eq. D; stencil PYCOOL_STENCIL_7PT, _ISO27 or _4TH) on every plane
 * wave exp(2 pi i m.x / n), m in numpy's FFT order ([z][y][x], x fastest);
 * values that follow their predecessor in the sorted list within 1e-12
 * (relative to max(1, |v|)) count as one -- a chain of such values joins one
 * group, so the tolerance is applied between neighbours, transitively.
 *   values (out, room for cap, may be NULL), ascending; count (out): how many;
 *   index (out, n^3 int32, may be NULL): each mode's position in values.
 * The host work holds 2 n^3 doubles (the symbols and a sorted copy).
 * E_INVALID: bad n (1..512) or stencil, count NULL, or cap too small. */
pycool_status pycool_linear_modes(int32_t n, int32_t stencil, double* values, int64_t cap,
                                  int64_t* count, int32_t* index);

/* The linearised evolution of lattice fields, end to end on the device
 * (Sec. 2.2, Eqs. phi-lin, Phik-1, pert-evo; Sec. 2.4: growth functions per
 * distinct k_eff^2, then a kernel that takes each Fourier position's matrix):
 *   1. the background phi0, pi0 = lattice means (fixed-order device sums) and
 *      the perturbations phi - phi0, pi - pi0 (Eq. phi-lin), written to
 *      phi_out, pi_out as scratch;
 *   2. forward real-to-complex FFTs of the perturbations (cuFFT), every
 *      field, their k = 0 coefficients cleared;
 *   3. the growth functions T of the distinct k_eff^2 values of the lattice's
 *      stencil, any of the three (pycool_linear_growth's kernel, background
 *      read on the device);
 *   4. every mode (dPhi, dPi)_k <- T[k_eff^2(k)] (dPhi, dPi)_k / n^3, and the
 *      k = 0 coefficient <- the evolved background;
 *   5. inverse FFTs into phi_out, pi_out: background(eta) + perturbations(eta).
 *   phi, pi (in) / phi_out, pi_out (out): device float64 [field][z][y][x],
 *     N_f n^3 values each; the inputs are not modified; outputs must not
 *     overlap the inputs.
 *   a0 > 0, pa0 (finite): the initial scale factor and its momentum (e.g. the
 *     p_a of pycool_energies for the same fields).
 *   background (out, host, 2 + 2 N_f doubles): a, p_a, phi0[N_f], pi0[N_f] at
 *     the end.
 * The call allocates its device work space (spectra, tables), works on
 * `cuda_stream` and synchronises it before returning.  The host tables of a
 * lattice size and the FFT plans of a (size, N_f, device) are kept for the
 * process's lifetime: the first call for a size pays for them, and calls that
 * share a plan run one at a time.
 * Errors: E_INVALID (bad config, n outside 2..512, bad pointers, or a
 * potential given at run time), E_NOMEM, E_CUDA.  The Q-ball's
 * second derivatives need |Phi0| > 0 throughout. */
pycool_status pycool_linear_evolve(const pycool_config* cfg, double a0, double pa0,
                                   const double* phi, const double* pi, int64_t steps,
                                   double* phi_out, double* pi_out, double* background,
                                   void* cuda_stream);

pycool_status pycool_linear_growth(const pycool_config* cfg, double a0, double pa0,
                                   const double* phi0, const double* pi0, const double* k2,
                                   int64_t nk, int64_t steps, double* T, double* background,
                                   void* cuda_stream);

/* Release the simulation and whatever the library allocated for it.  Waits for
 * the simulation's queued work first.  NULL is ignored. */
void pycool_destroy(pycool_sim* sim);

/* Static description of a status code. */
const char* pycool_strerror(pycool_status status);
/* ---- serving: many simulations resident on one GPU ---------------------------
 * The paper's multi-simulation use (Sec. 2.4: Delta-N from many runs with
 * different initial values; Sec. 4: many lattices evolved simultaneously) as
 * a continuous-batching server.  A server thread admits queued requests while
 * the HBM budget and slot count allow, generates their initial fields on the
 * device, and advances every resident simulation that shares a kernel instance
 * with one launch per stage (CUDA graphs of several stages, rebuilt when the
 * membership changes).  A request's result is bit-identical whether it ran
 * alone or with others. */

/* Initial-condition recipes generated on the device.  WHITE:
 *   phi_i = background_i + noise N(0,1),  pi_i = momentum_i + noise N(0,1),
 * with the normals from Philox4x32-10 (Salmon et al., SC'11), key = seed,
 * counter = (e/4, array, 0, 0) for element e of array phi_1..phi_N, pi_1..pi_N,
 * and Box-Muller on the uniforms (x + 1/2) 2^-32 (component e mod 4). */
typedef enum { PYCOOL_IC_WHITE = 0 } pycool_ic_kind;

typedef struct {
  double background[PYCOOL_MAX_FIELDS];
  double momentum[PYCOOL_MAX_FIELDS];
  double noise;     /* rms of the white noise, >= 0                        */
  double a0;        /* initial scale factor (<= 0 means 1)                 */
} pycool_ic;

/* Start a server that keeps up to max_slots simulations resident and reserves
 * hbm_budget bytes of device memory for them (one arena, allocated here).
 * The server owns one host thread and its own CUDA streams on the device that
 * is current at this call.  E_NOMEM if the arena cannot be reserved. */
pycool_status pycool_server_create(size_t hbm_budget, int32_t max_slots, pycool_server** out);

/* Queue a simulation (cfg, initial-condition recipe, RNG seed, time steps);
 * *ticket identifies it.  E_INVALID / E_UNSTABLE_DT for a bad config, E_NOMEM if
 * it could never fit the budget.  Thread-safe; never blocks on the GPU. */
pycool_status pycool_server_submit(pycool_server* srv, const pycool_config* cfg,
                                   const pycool_ic* ic, uint64_t seed, int64_t steps,
                                   uint64_t* ticket);

/* Wait (at most timeout_s seconds; < 0 = no limit) for a ticket's result: the
 * observables of its final, synchronised state.  Returns the run's status
 * (OK, E_NONFINITE, ...), E_TIMEOUT if not finished in time (the ticket stays
 * valid), E_NOT_FOUND for an unknown or already collected ticket.  Thread-safe. */
pycool_status pycool_server_wait(pycool_server* srv, uint64_t ticket, double timeout_s,
                                 pycool_observables* out);

/* Latency percentiles (submission to result, seconds) of the completed
 * requests, the aggregate site-updates per second between the first admission
 * and the last completion, and the number of completed requests. */
pycool_status pycool_server_stats(pycool_server* srv, double* p50_s, double* p99_s,
                                  double* site_updates_per_s, int64_t* completed);

/* Cancel a request.  A queued request is dropped at once; a resident one is
 * retired at the server's next graph boundary (its launches complete first,
 * its memory returns to the arena).  wait() then returns E_CANCELLED with the
 * observables of the state it reached (all zero if it was never admitted).
 * Returns OK, E_NOT_FOUND for an unknown or collected ticket, E_STATE if the
 * request has finished already (collect it with wait).  Thread-safe. */
pycool_status pycool_server_cancel(pycool_server* srv, uint64_t ticket);

/* Which requests run on the persistent kernel (the one-launch-per-evolve
 * stepper of pycool_evolve, Sec. 2.3) instead of the per-stage launches they
 * share with the other members of their group: FP64 requests whose side n is a
 * multiple of 32 and at least min_n (0: none; default 256).  Such a member gets
 * one cooperative launch of up to one graph's worth of stage sweeps (8) at
 * each graph boundary, alone on the GPU: a cooperative grid holds every SM.
 * Its launches leave the stage boundary pending, as the per-stage launches do;
 * its last launch ends with the flush.  Applies to requests admitted after the
 * call; the path a request takes depends on its config and min_n only, so
 * results stay identical alone and in a mix.  E_INVALID unless min_n is 0 or a
 * multiple of 32.  Thread-safe. */
pycool_status pycool_server_set_persistent_min_n(pycool_server* srv, int32_t min_n);

/* Stop the server thread and release every resident simulation and the arena. */
void pycool_server_destroy(pycool_server* srv);

/* ---- fault injection (tests of failure detection) ----------------------------
 * Failures are made on the host or through a bounded device-side wait; nothing
 * here traps or faults the GPU.  The paper has no counterpart.
 *
 * pycool_debug_fail_alloc: the next `count` device allocations the library
 *   makes (pycool_create with NULL buffers, pycool_server_create's arena)
 *   report failure as an exhausted cudaMalloc would: the call returns E_NOMEM
 *   and leaves nothing allocated.  count = 0 clears it.  Process-wide.
 * pycool_debug_barrier_stall: the simulation's next persistent launch (the
 *   next pycool_evolve of a lattice with n a multiple of 32) waits at its
 *   first grid barrier for one block more than the launch has -- an arrival
 *   that never comes -- with every device-side wait limited to
 *   wait_limit_clocks SM clocks.  Every block gives up at the limit, records
 *   the fault and returns; pycool_sync then returns E_TIMEOUT and the
 *   simulation is poisoned (E_STATE) while the CUDA context stays usable.
 *   E_STATE if the simulation does not use the persistent kernel. */
pycool_status pycool_debug_fail_alloc(int32_t count);
pycool_status pycool_debug_barrier_stall(pycool_sim* sim, int64_t wait_limit_clocks);

/* ---- allocation-free stage sweep ---------------------------------------------
 * The paper has no counterpart to this call; it is a deployment convenience.
 *
 * For callers that cannot call cudaMalloc: code whose device memory belongs to
 * another allocator (a framework's caching allocator, a pre-reserved arena
 * that leaves nothing for cudaMalloc) and host loops that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree may cause.  The caller owns
 * the field arrays; every other byte the sweep needs (background record,
 * launch descriptor, per-block partial sums, ticket) lives in one file-scope
 * device array of PYCOOL_NOALLOC_SCRATCH_BYTES, which every GPU that loads the
 * library holds until the process exits.  No call here allocates.
 *
 * One call = one launch of the FP64 stage sweep of pycool_evolve:
 *   flush == 0 : the fused sweep of stage `state->stage` (drift merged with the
 *                pending half-stage, Laplacian, kick); reads phi_in, pi_in,
 *                writes phi_out and pi_out.  The result is staggered
 *                (state->h_prev != 0), as between the sweeps of pycool_evolve.
 *   flush != 0 : the synchronising drift; reads phi_in, pi_in, writes phi_out
 *                (pi is unchanged: use pi_in as the momentum; pi_out unused)
 *                and fills state->obs.  With h_prev == 0 it only reduces
 *                (phi_out becomes a copy of phi_in): start every run with such
 *                a call, state->init_pa = 1 sets p_a from H = 0.
 * A time step of order 2, 4, 6, 8 is 1, 3, 7, 15 non-flush calls; the caller
 * swaps its two buffer pairs between calls.  Arrays: float64 device memory,
 * [field][z][y][x], 16-byte aligned; config precision must be PYCOOL_FP64.
 *
 * Errors: E_INVALID for a bad config, bad pointers, an output array that
 * shares memory with an input array or with the other output (the sweep reads
 * neighbours of the inputs while it writes the outputs), init_pa set on a
 * non-flush call, or a lattice whose sweep needs more than
 * pycool_noalloc_max_blocks() blocks (about n <= 512 for two fields);
 * E_NONFINITE if a sum overflowed; E_CUDA / E_TIMEOUT as elsewhere.
 * The call synchronises the stream (it reads the background record back).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every call
 * shares the one array and it keeps the last call's contents (the call clears
 * what must start at zero): calls whose work overlaps on the GPU, from two
 * streams or two threads, race and must not be issued. */
#define PYCOOL_NOALLOC_SCRATCH_BYTES (1u << 20)

typedef struct {
  double a, pa, eta;      /* scale factor, its momentum, conformal time             */
  double h_prev;          /* pending half-stage step (0 = synchronised)             */
  double sum_pi2;         /* sum of pi^2 of the current momentum                    */
  int64_t stage;          /* stage-table index of the next sweep                    */
  int64_t steps_done;     /* completed time steps                                   */
  int32_t init_pa;        /* in: 1 = the next flush sets p_a from H = 0             */
  int32_t error;          /* out: 1 = a lattice sum was not finite                  */
  pycool_observables obs; /* out, flush calls: observables of the synchronised state */
} pycool_stage_state;

/* Largest number of blocks (lattice tiles x z-chunks) a sweep may use here. */
size_t pycool_noalloc_max_blocks(void);

pycool_status pycool_sweep_noalloc(const pycool_config* cfg, const double* phi_in,
                                   const double* pi_in, double* phi_out, double* pi_out,
                                   int32_t flush, pycool_stage_state* state, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PYCOOL_H */
