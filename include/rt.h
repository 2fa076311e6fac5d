/*
 * rtgb: GB300 (sm_103a) radiative-transfer step of the M1 moment method
 * (Rosdahl et al. 2013, "RAMSES-RT"), on a uniform Cartesian grid.
 *
 * One RT step over a time step dt is, in order (paper Sec. 3):
 *   1. injection       N_i += L_i dt / V in each source cell    (Sec. 3.1, Eq. (injnum))
 *   2. transport       explicit first-order Godunov update of (N_i, F_i)
 *                      with the M1 closure and GLF or HLL intercell fluxes,
 *                      unsplit over the six faces          (Sec. 3.2, Eqs. (dUdt_sol),
 *                                                          (hll), (glf); Sec. 2, Eqs. (edd2)-(Udir))
 *   3. thermochemistry per-cell semi-implicit update of N_i, F_i, T, x_HII,
 *                      x_HeII, x_HeIII, sub-cycled under the 10% rule
 *                                                          (Sec. 3.3, App. A)
 * with dt bounded by the Courant condition dt <= CFL dx / (3 c_r)
 * (Sec. 4.1, Eq. (dt_courant)) and c_r the reduced speed of light.
 *
 * Units are cgs.  Layouts (x fastest, row-major, no padding):
 *   scalar fields      [nz][ny][nx]                 (cells = nx*ny*nz)
 *   photon density N   [G][nz][ny][nx]              photons / cm^3
 *   photon flux F      [G][3][nz][ny][nx]           photons / cm^2 / s  (x, y, z)
 *   group constants    sigN, sigE [G][3] cm^2 (species HI, HeI, HeII), egy [G] erg
 *
 * Ownership: the handle owns all device memory it allocates.  Every input
 * is copied at the call; every get_* copies into caller buffers.  With
 * device_ptrs = 1, pointers are CUDA device pointers on the handle's device
 * and are read/written on the handle's stream.
 *
 * Errors: every int-returning call returns RT_OK (0) or a negative code.
 * Device-side failures (sub-cycle cap, queue overflow, non-finite values)
 * set a sticky status word that the next rt_step / rt_get_* / rt_sync
 * reports as its return code; the state is then undefined until
 * rt_set_state.  rt_last_error gives a one-line message.
 */
#ifndef RTGB_RT_H
#define RTGB_RT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_OK 0
#define RT_EINVAL -1     /* bad sizes / options / non-finite or out-of-range inputs */
#define RT_EDT -2        /* dt above the Courant limit */
#define RT_ESUBCYCLE -3  /* a cell exceeded max_subcycles thermochemistry attempts */
#define RT_EQUEUE -4     /* work-queue overflow */
#define RT_ECUDA -5      /* a CUDA runtime call failed */
#define RT_ENOMEM -6     /* device or host allocation failed */
#define RT_ENONFINITE -7 /* a NaN/Inf appeared in the state */

#define RT_MAX_GROUPS 8

enum { RT_BC_OUTFLOW = 0, RT_BC_REFLECT = 1, RT_BC_PERIODIC = 2, RT_BC_INFLOW = 3 };
enum { RT_GLF = 0, RT_HLL = 1 };
enum { RT_FP64 = 0, RT_MIXED = 1, RT_MIXED32 = 2 };
#define RT_REC_BY_BAND -2

typedef struct rt_handle rt_handle;

/* Uniform grid.  bc[] = boundary condition of the faces -x, +x, -y, +y, -z,
 * +z: outflow (zero-gradient ghost), reflect (ghost with the normal flux
 * component negated), periodic, or inflow (a ghost held at a given photon
 * state, rt_set_inflow; zero until set; single-box handles only), e.g.
 * the constant flux entering the box of the paper's Sec. 6 test 3. */
typedef struct {
    int nx, ny, nz;
    double dx_cm;
    int bc[6];
} rt_grid;

/* Options.  X: hydrogen mass fraction (Y = 1 - X; helium is skipped when
 * Y = 0).  isothermal: T held fixed.  otsa: on-the-spot approximation
 * (case-B rates, no recombination photons; Sec. 3.3.2; default 1).
 * flux: RT_GLF (default) or RT_HLL.  cfl: Courant factor (0.8).
 * precision: RT_FP64; RT_MIXED (photon state and transport in FP32 with
 * compensated face sums, thermochemistry in FP64); RT_MIXED32 (as
 * RT_MIXED, with the exponentials of the rate fits and the absorption
 * coefficients of the thermochemistry in FP32, the fits' arguments in
 * float pairs and its updates in FP64).  a_exp: expansion
 * factor in the Compton term (1).  max_subcycles: thermochemistry attempts
 * allowed per cell and step (1e6).  smooth: 0, or 1 for smoothed RT (Sec.
 * 3.4): the change of N_i, F_i over injection and transport enters the
 * thermochemistry as the rates (N'_i - N^t_i)/dt, (F'_i - F^t_i)/dt of its
 * photon update, which starts from the state before injection
 * (Eqs. (smoothrate1), (smoothrate2)); single-box handles only (the batch,
 * the adjoint and rt_thermo_step_noalloc take 0).  otsa = 0 (single-box
 * handles only): case-A rates and recombination photons
 * C_i = sum_j b_ji (alpha^A_j - alpha^B_j) n_j n_e (Eqs. (thchem_N),
 * (cool_N_cr)); rec_group[j] is the group that recombinations of HII,
 * HeII, HeIII emit into, -1 for none, RT_REC_BY_BAND (the default) for
 * group min(j, G - 1) (groups ordered by band); the budget's absorbed
 * column is then absorbed minus created. */
typedef struct {
    double X;
    int isothermal;
    int otsa;
    int flux;
    double cfl;
    int precision;
    double a_exp;
    int max_subcycles;
    int smooth;
    int rec_group[3];
} rt_options;

/* Fill *o with the defaults listed above (X = 0.76). */
void rt_default_options(rt_options *o);

/* Create a handle on the current CUDA device.  n_groups in 1..RT_MAX_GROUPS,
 * c_r > 0 the reduced light speed [cm/s]; sigN, sigE [G][3] group cross
 * sections (Eqs. (csn_multi), (cse_multi)) and egy [G] mean photon energies
 * (Eq. (egy_multi)), host pointers, copied.  The state starts at zero
 * photons, n_H = 0, and must be set with rt_set_state before rt_step. */
int rt_create(const rt_grid *grid, int n_groups, const rt_options *opt, double c_r,
              const double *sigN, const double *sigE, const double *egy, rt_handle **out);

/* Free the handle and all its device memory.  NULL is allowed. */
void rt_destroy(rt_handle *h);

/* Use `stream` (a cudaStream_t, may be NULL for the legacy default stream)
 * for all later work of this handle. */
int rt_set_stream(rt_handle *h, void *stream);

/* Set the full state (all pointers required).  nH > 0; x_HII in
 * [1e-6, 1]; x_HeII, x_HeIII >= 0 with sum <= 1; T > 0; N >= 0;
 * |F| <= c_r (N (1 + 1e-8) + 1e-290) (the slack covers sub-normal
 * photon densities left by strong absorption).  Validated on the host for host pointers;
 * device pointers are copied without validation.  Resets the budget. */
int rt_set_state(rt_handle *h, const double *nH, const double *xHII, const double *xHeII,
                 const double *xHeIII, const double *T, const double *N, const double *F,
                 int device_ptrs);

/* Copy the state out; any pointer may be NULL to skip that field.
 * Synchronises the handle's stream and reports sticky device errors. */
int rt_get_state(rt_handle *h, double *nH, double *xHII, double *xHeII, double *xHeIII,
                 double *T, double *N, double *F, int device_ptrs);

/* Replace the point-source list: n sources, ijk [n][3] = (i, j, k) cell
 * indices (x, y, z), L [n][G] photons/s, host pointers.  Sources sharing a
 * cell are merged (luminosities summed in the given order). */
int rt_set_sources(rt_handle *h, int n, const int32_t *ijk, const double *L);

/* Ghost state of an RT_BC_INFLOW face (0..5 = -x, +x, -y, +y, -z, +z):
 * state [G][4] = (N photons/cm^3, Fx, Fy, Fz photons/cm^2/s) per group,
 * host pointer, copied; |F| <= c_r N required.  RT_EINVAL if the face is
 * not an inflow face or the state is not realisable. */
int rt_set_inflow(rt_handle *h, int face, const double *state);

/* Change the expansion factor to a (Sec. 5, cosmological settings).  The
 * photons are kept in the super-comoving variables N~ = a^3 N,
 * F~ = a^4 F / (H0 L) and the gas at constant comoving density, so the
 * physical N, F and n_H held by the handle scale by (a_old/a)^3,
 * (a_old/a)^4 and (a_old/a)^3; the physical cell width becomes
 * dx * a / a_old and the Compton term takes T_gamma = 2.727 / a.  Between
 * two changes the super-comoving transport equations are the physical
 * ones at that cell width, so rt_step is unchanged (the Courant dt follows
 * dx).  a_old is the previous value, initially rt_options.a_exp.  The
 * adiabatic cooling of the gas is not applied (it belongs to the
 * hydrodynamics).  Needs a state; enqueued on the handle's stream. */
int rt_set_scale_factor(rt_handle *h, double a);

/* Courant time step CFL dx / (3 c_r), Eq. (dt_courant). */
int rt_courant_dt(const rt_handle *h, double *dt);

/* One RT step (injection, transport, thermochemistry, budget) of length
 * dt; dt <= 0 takes the Courant step; dt above it returns RT_EDT.
 * Asynchronous on the handle's stream. */
int rt_step(rt_handle *h, double dt);

/* nsteps RT steps of length dt (as rt_step), launched as a CUDA graph
 * captured once per (dt, source list). */
int rt_run(rt_handle *h, double dt, int nsteps);

/* Photon budget per group, out [G][4]: photons in the box now, and since
 * the last rt_set_state the photons absorbed by the gas, the net outflow
 * through the box faces (negative = inflow), and the photons emitted by
 * the sources.  Conservation: in_box(now) = in_box(at set_state) +
 * emitted - absorbed - outflow, up to rounding.  Synchronises. */
int rt_get_budget(rt_handle *h, double *out);

/* Thermochemistry attempts (successful and rejected thermo_step calls) of
 * each cell in the last step, [nz][ny][nx] int32.  Synchronises. */
int rt_get_subcycles(rt_handle *h, int32_t *per_cell, int device_ptr);

/* Wait for the handle's stream and report sticky device errors. */
int rt_sync(rt_handle *h);

/* One-line description of the last error on this handle (never NULL). */
const char *rt_last_error(const rt_handle *h);

/* ---- adjoint (vector-Jacobian products of rt_step) ----
 *
 * The adjoint of the step U_k -> U_{k+1} of rt_step (injection, transport,
 * thermochemistry, in the paper's order, Sec. 3): given lambda = dJ/dU_{k+1}
 * for a scalar J, it returns lambda = dJ/dU_k and accumulates dJ/dn_H and
 * dJ/dL.  The thermochemistry is differentiated along the sub-cycle
 * schedule that the forward step takes (the schedule is piecewise constant
 * in the inputs, so this is the derivative wherever it exists), the
 * transport is the transposed GLF or HLL stencil of the handle's flux
 * (with HLL, the derivative of the tabulated wave speeds included; where
 * two cells' speeds tie exactly the step has a kink and the derivative is
 * that of the branch max/min selects).  Needs precision RT_FP64, the OTSA
 * and smooth = 0 (else RT_EINVAL), flux RT_GLF or RT_HLL, and a state
 * set by rt_set_state.
 *
 * All arrays are CUDA device pointers on the handle's device, used on the
 * handle's stream, in the state layouts above:
 *   lam_xHII, lam_xHeII, lam_xHeIII, lam_T  [cells]        in: dJ/dU_{k+1}, out: dJ/dU_k
 *   lam_N [G][cells], lam_F [G][3][cells]                  in/out likewise
 *   g_nH  [cells]                                          += dJ/dn_H of the step
 *   g_L   [n][G]  (n, order: the last rt_set_sources)      += dJ/dL (s photons/s)^-1
 * dt <= 0 means the Courant dt.  The handle's state is left at U_k; the
 * budget and sub-cycle counts afterwards are those of recomputed steps.
 * mismatches: NULL, or a host counter to which the number of cells whose
 * recomputed attempt count differs from the forward kernels' is added (this
 * re-runs the forward thermochemistry on a copy and synchronises; nonzero
 * means the adjoint differentiated another schedule than the forward run). */
int rt_step_vjp(rt_handle *h, double dt, double *lam_xHII, double *lam_xHeII, double *lam_xHeIII, double *lam_T,
                double *lam_N, double *lam_F, double *g_nH, double *g_L, long long *mismatches);

/* nsteps steps of rt_step_vjp from the handle's state U_0: recomputes and
 * keeps the forward trajectory U_0..U_{nsteps-1} on the device (nsteps x
 * (4 + 4G) x cells doubles, allocated for the call), then sweeps it back;
 * lambda goes in as dJ/dU_nsteps and comes out as dJ/dU_0.  The handle ends
 * at U_0.  Synchronises. */
int rt_run_vjp(rt_handle *h, double dt, int nsteps, double *lam_xHII, double *lam_xHeII, double *lam_xHeIII,
               double *lam_T, double *lam_N, double *lam_F, double *g_nH, double *g_L, long long *mismatches);

/* Host-side HLL wave-speed table used by RT_HLL: extreme eigenvalues of the
 * M1 flux Jacobian (Sec. 3.2) in units of c, out [nf][nmu][2] =
 * (lambda_min, lambda_max) at f = k/(nf-1), mu = -1 + 2j/(nmu-1).
 * Needs no GPU. */
int rt_hll_table(int nf, int nmu, double *out);

/* Routing of the thermochemistry (tuning and tests; no counterpart in the
 * paper).  The sub-cycling of Sec. 3.3.1 runs in up to four kernels per
 * step: a first pass (one thread per cell, pass1_attempts attempts), a
 * lane-per-cell drain of the cells still sub-cycling (drain_budget more
 * attempts each), a second such drain (drain2_budget) that runs only when
 * more than drain2_min_cells cells are left for it, and a pair of warps
 * per cell for the rest.  Routing decides which kernel runs which attempts
 * of a cell, never the arithmetic of an attempt: x_HII, x_HeII, x_HeIII, T,
 * N, F and the attempt counts are identical for every routing (a queued
 * cell carries its flux scale prod 1/(1 + h D_i), and F is formed once,
 * when the cell finishes).  Values <= 0
 * (drain2_min_cells < 0) restore the defaults 6, 128, 128 and eight cells
 * per warp of the tail kernel.  Takes effect at the next step. */
int rt_set_thermo_routing(rt_handle *h, int pass1_attempts, int drain_budget, int drain2_budget,
                          long long drain2_min_cells);

/* Per-phase timing (diagnostics; not part of the RT method).  With enable
 * != 0, rt_step records CUDA events on the handle's stream around each of
 * its phases (rt_run does not).  Phases: 0 injection, 1 transport,
 * 2 thermochemistry first pass, 3 thermochemistry queue drain, 4 photon
 * reduction, 5 budget finalisation.  Enabling resets the counters. */
#define RT_NPHASES 6
int rt_set_profiling(rt_handle *h, int enable);

/* Accumulated milliseconds and launch counts per phase since profiling was
 * enabled, ms [RT_NPHASES], launches [RT_NPHASES].  Synchronises. */
int rt_get_profile(rt_handle *h, double *ms, int64_t *launches);

/* ---- Batched boxes ----
 * Many independent boxes of uneven sizes advanced together: each box runs
 * exactly the RT step above on its own grid, state, sources and photon
 * groups; all boxes share the cell width dx_cm, the reduced light speed and
 * the options, hence one Courant step.  Boxes with the same number of
 * groups must share the group constants.  Every phase of a step covers all
 * boxes in one launch per tile shape / group count, and rt_batch_run
 * replays a step pair as a CUDA graph. */
typedef struct rt_batch rt_batch;

/* n_boxes grids (all with the same dx_cm), n_groups[b] in 1..RT_MAX_GROUPS,
 * sigN[b], sigE[b] ([G_b][3] cm^2) and egy[b] ([G_b] erg) host pointers per
 * box.  Returns RT_EINVAL for bad sizes, mixed dx or differing constants
 * within a group count. */
int rt_batch_create(int n_boxes, const rt_grid *grids, const int *n_groups, const rt_options *opt, double c_r,
                    const double *const *sigN, const double *const *sigE, const double *const *egy,
                    rt_batch **out);
void rt_batch_destroy(rt_batch *b);
int rt_batch_set_stream(rt_batch *b, void *stream);
/* State of box `box` in the single-box layout of that box (see rt_set_state);
 * restarts that box's budget. */
int rt_batch_set_box_state(rt_batch *b, int box, const double *nH, const double *xHII, const double *xHeII,
                           const double *xHeIII, const double *T, const double *N, const double *F,
                           int device_ptrs);
int rt_batch_get_box_state(rt_batch *b, int box, double *nH, double *xHII, double *xHeII, double *xHeIII,
                           double *T, double *N, double *F, int device_ptrs);
/* Sources of box `box` (cell indices within the box), as rt_set_sources. */
int rt_batch_set_box_sources(rt_batch *b, int box, int n, const int32_t *ijk, const double *L);
int rt_batch_courant_dt(const rt_batch *b, double *dt);
int rt_batch_step(rt_batch *b, double dt);
int rt_batch_run(rt_batch *b, double dt, int nsteps);
/* Budget of box `box`, out [G_b][4] as rt_get_budget.  Synchronises. */
int rt_batch_get_budget(rt_batch *b, int box, double *out);
int rt_batch_sync(rt_batch *b);
const char *rt_batch_last_error(const rt_batch *b);
/* Times the transport of each distinct box shape with 32x8 and 16x16 tiles
 * and 4, 8, 16 or 32 planes per CTA (`trials` launches each, on the current
 * state, which it does not change) and keeps the fastest.  Synchronises. */
int rt_batch_autotune(rt_batch *b, int trials);
/* Tiling chosen for a box: shape 0 = 32x8, 1 = 16x16; planes per CTA. */
int rt_batch_box_tiling(const rt_batch *b, int box, int *shape, int *planes);

/* Allocation-free thermochemistry (no counterpart in the paper): the
 * sub-cycled thermochemistry of one RT step (what rt_step does after the
 * transport) applied in place to caller-owned device arrays, for callers
 * that cannot allocate device memory at call time, such as code running
 * under another framework that has reserved all device memory for its own
 * pool, or a loop with a fixed memory footprint that must not call into
 * the CUDA allocator.  No handle is needed and nothing is allocated: the
 * work queue lives in a fixed device array of the library, sized for at
 * most 262144 cells (29.4 MB held on every GPU that loads the library until
 * the process exits).  ncells above that returns RT_EINVAL, as do the
 * option values rt_create rejects.
 * Arguments: ncells cells in any order (one value per cell), the options,
 * c_r and group constants as for rt_create (host pointers), dt > 0; nH,
 * xHII, xHeII, xHeIII, T [ncells], N [G][ncells], F [G][3][ncells] and
 * subcycles [ncells] (attempts per cell, written) are device pointers on
 * the current device, updated in place on `stream` (a cudaStream_t, NULL =
 * legacy default stream).  The call waits for the stream and returns
 * RT_OK or the device status (RT_ESUBCYCLE, RT_EQUEUE, RT_ENONFINITE);
 * RT_ECUDA if a CUDA call fails.
 * The first call on each device looks up the array's device address with
 * that device current (the device must be current when calling); make that
 * first call before any stream capture.  After a device reset (a new
 * primary context, hence a new copy of the array) the next call looks the
 * address up again.  Every call uses the same array and clears its
 * counters first; calls that overlap on the GPU race on it. */
int rt_thermo_step_noalloc(long long ncells, int n_groups, const rt_options *opt, double c_r,
                           const double *sigN, const double *sigE, const double *egy, double dt,
                           const double *nH, double *xHII, double *xHeII, double *xHeIII,
                           double *T, double *N, double *F, int32_t *subcycles, void *stream);

/* The exp (fn 0), log (fn 1), log1p (fn 2), reciprocal (fn 3), square
 * root (fn 4), softplus ln(1 + e^x) (fn 5) and its derivative 1/(1 + e^-x)
 * (fn 6) that the library's FP64 rate fits use (double-float arithmetic on
 * float pairs, table-driven exp and log after Tang 1989/1990, piecewise
 * interpolating polynomials for softplus), applied to n doubles:
 * y[i] = f(x[i]); x, y device pointers,
 * enqueued on `stream` (NULL: the default stream), no synchronisation.
 * For accuracy checks against CUDA's own functions.  RT_EINVAL for a bad
 * fn or null arrays. */
int rt_fmath_eval(int fn, long long n, const double *x, double *y, void *stream);

/* Host-side copy of the thermochemistry's rate functions (App. A rate
 * fits, Cen 1992, Hui & Gnedin 1997, Black 1981, the cooling terms of Eq.
 * (rate_cooling)), each evaluated on the GPU as
 *     f(T) = Cc exp(c0 + c1 ln T + c2 / T - c3 ln(1 + exp(c4 ln T + c5))):
 * out [32][7] = (Cc, c0, c1, c2, c3, c4, c5) per slot, the constants as the
 * kernels hold them (c0..c5 as the sums of their float pairs).  Slots 0..10:
 * the cooling terms zeta_HI, psi_HI, eta_HII, theta, zeta_HeI, zeta_HeII,
 * psi_HeII, eta_HeII, the two omega_HeII terms, eta_HeIII (erg cm^3 s^-1,
 * times their density); 16..21: beta_HI, alpha_HII, beta_HeI, beta_HeII,
 * alpha_HeII, alpha_HeIII (cm^3 s^-1); the others zero.  case_b: 1 the
 * case-B recombination fits, 0 case A.  Needs no GPU.  RT_EINVAL for a bad
 * case or a null out. */
int rt_rate_functions(int case_b, double *out);

/* Library version (major * 10000 + minor * 100 + patch). */
int rt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RTGB_RT_H */
