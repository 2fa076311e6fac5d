// Internal definitions shared by the rtgb translation units (not part of the
// C-ABI).  Device kernels live in transport.cu, thermo.cu and misc.cu; the
// C-ABI in rt_api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rt.h"

namespace rtgb {

constexpr int kMaxG = RT_MAX_GROUPS;
constexpr int kHllNF = 257;   // HLL table: f = k/256
constexpr int kHllNMU = 257;  // mu = -1 + j/128

// Sticky device status bits.
enum : unsigned {
    kStatusSubcycle = 1u,
    kStatusQueue = 2u,
    kStatusNonFinite = 4u,
};

// Constants of the photon groups, passed by value to the kernels.
struct GroupConsts {
    double sigN[kMaxG][3];   // cm^2, species HI, HeI, HeII
    double sigE[kMaxG][3];   // cm^2
    double egy[kMaxG];       // erg
};

struct GridDev {
    int nx, ny, nz;
    long long nc;            // cells
    long long stride;        // distance between consecutive groups / flux components
    double dx;               // cm
    int bc[6];
};

// Batched boxes: a box of a group-count class, and one CTA's work item.
struct BatchBox {
    GridDev g;               // g.stride = cells of the box's class
    long long cell_off;      // first cell of the box within its class
    int cls;                 // class index (boxes with the same G)
    int G;
};
struct BatchItem {
    int box, grp;
    int x0, y0, z0, z1;
};

// Parameters of the thermochemistry kernels.
struct ThermoParams {
    long long nc;
    double dt;               // RT step
    double cr;               // reduced light speed
    double X;                // hydrogen mass fraction
    double he_ratio;         // n_He / n_H = Y / (4 X)
    double kfac;             // (gamma - 1) X / k_B, so K = kfac / n_H
    double a_exp;
    int isothermal;
    int helium;              // Y > 0
    int case_b;
    int max_sub;
    int pass1_attempts;      // attempts before a cell is handed to the queue
    int drain_budget;        // attempts a cell may spend in the first lane-per-cell drain
    int drain2_budget;       // ... and in the second
    long long drain2_min;    // the second drain runs only above this many queued cells
                             // (< 0: eight per warp of the warp-per-cell kernel)
    int emit;                // no OTSA: recombination photons (Sec. 3.3.2)
    int rec_g[3];            // group receiving HII, HeII, HeIII recombination photons (-1: none)
    GroupConsts gc;
    // derived per-group terms of the photon update (derive_group_terms):
    double crs[kMaxG][3];    // c_r sigma^N_ij, the absorption coefficient per absorber
    double hq[kMaxG][3];     // egy_i sigma^E_ij - eps_j sigma^N_ij, photoheating per absorber
    double tg;               // T_gamma = 2.727 / a, the Compton temperature
    double comp;             // 1.017e-37 T_gamma^4, Compton exchange per (T - T_gamma) n_e
};

// Fill ThermoParams::crs and ::hq from cr and gc (the photoheating term of
// Eq. (PHeat2): each absorbed photon of group i heats by its mean energy
// minus the ionisation energy eps_j of the absorber, 13.60, 24.59, 54.42 eV),
// and the Compton constants from a_exp.  Call after setting cr, gc, a_exp.
inline void derive_group_terms(ThermoParams &p)
{
    const double ev = 1.602176634e-12;
    const double eps[3] = {13.60 * ev, 24.59 * ev, 54.42 * ev};
    for (int i = 0; i < kMaxG; ++i)
        for (int j = 0; j < 3; ++j) {
            p.crs[i][j] = p.cr * p.gc.sigN[i][j];
            p.hq[i][j] = p.gc.egy[i] * p.gc.sigE[i][j] - eps[j] * p.gc.sigN[i][j];
        }
    // Compton cooling/heating of the rate appendix, varpi = 1.017e-37 T_g^4 (T - T_g)
    p.tg = 2.727 / p.a_exp;
    p.comp = 1.017e-37 * (p.tg * p.tg * p.tg * p.tg);
}

// Default routing of cells between the thermochemistry kernels.  Routing
// decides only which kernel runs which attempts of a cell, never the
// arithmetic of an attempt.
inline void default_routing(ThermoParams &p)
{
    p.pass1_attempts = 6;
    p.drain_budget = 128;
    p.drain2_budget = 128;
    p.drain2_min = -1;
}

// Device work queues of cells whose sub-cycling outlasted the first pass
// (a) and the lane-per-cell drain (b); queue c, the input of the
// warp-per-cell kernel, reuses the arrays of a once a is drained.
constexpr int kQueueCounters = 8;

struct QueueArrays {
    uint32_t *cell;
    double *t_left;
    double *dt_tc;
    int32_t *attempts;
};
struct Queue {
    QueueArrays a, b;
    unsigned long long *counters;   // kQueueCounters: [0] a.count, [1] a.head, [2] b.count,
                                    // [3] b.head, [4] c.count, [5] c.head
    long long capacity;             // items per queue
    double *fscale;                 // [2G][nc]: a queued cell's flux scale Fs_i (rows 0..G-1) and,
                                    // smoothed RT, its Fdot weight Fb_i (rows G..2G-1)
};

// Per-block partial sums of the photon budget.
struct Partials {
    double *tr_inbox;     // [G][n_tr_blocks]  sum N after transport
    double *tr_outflow;   // [G][n_tr_blocks]  net outflow in the step
    double *th_inbox;     // [G][n_red_blocks] sum N after thermochemistry
    int n_tr_blocks;      // per group
    int n_red_blocks;     // per group
};

// ---- launchers (defined in the .cu files) ----
// transport: reads N0/F0, writes N1/F1 for all groups.  inflow: NULL, or
// the ghost states [G][6 faces][N, Fx, Fy, Fz] of RT_BC_INFLOW faces.
cudaError_t launch_transport(const GridDev &g, int G, int flux, double cr, double dt,
                             const double *N0, const double *F0, double *N1, double *F1,
                             const double *hll_table, const double *inflow, const Partials &p, cudaStream_t s);
// FP32 state (RT_MIXED): same scheme, compensated update.
cudaError_t launch_transport_f32(const GridDev &g, int G, int flux, double cr, double dt, const float *N0,
                                 const float *F0, float *N1, float *F1, const float *hll_table,
                                 const float *inflow, const Partials &p, cudaStream_t s);
// CTAs of the single-box transport launch (persistent: a fixed number per
// SM), and so the budget partials per group
int transport_grid(int n_sm, bool fp32);
// Batched transport over items [item0, item0 + nitems) of one tile shape
// (0: 32 x 8, 1: 16 x 16); N0/F0/N1/F1 are device arrays of per-class base
// pointers; partials are indexed by item.
cudaError_t launch_transport_batch(const BatchItem *items, const BatchBox *boxes, int item0, int nitems,
                                   int shape, bool fp32, int flux, double cr, double dt, double dx,
                                   const void *const *N0, const void *const *F0, void *const *N1,
                                   void *const *F1, const void *tab, double *pin, double *pout, cudaStream_t s);
// ... all items of both tile shapes in one launch (items [0, n_shape0) of
// shape 0, the rest of shape 1)
cudaError_t launch_transport_batch_all(const BatchItem *items, const BatchBox *boxes, int n_shape0, int nitems,
                                       bool fp32, int flux, double cr, double dt, double dx, const void *const *N0,
                                       const void *const *F0, void *const *N1, void *const *F1, const void *tab,
                                       double *pin, double *pout, cudaStream_t st);
void transport_init();   // kernel attributes; called once per handle

// ev (optional, 4 events): recorded around the first pass (0, 1) and
// around the queue drains (2, 3).  Npre, Fpre: NULL, or smoothed RT (Sec.
// 3.4): the photon state before injection and transport, N, F the state
// after them; both pairs are overwritten.
cudaError_t launch_thermo(const ThermoParams &tp, int G, const double *nH, double *xHII,
                          double *xHeII, double *xHeIII, double *T, double *N, double *F,
                          double *Npre, double *Fpre, int32_t *subcycles, Queue q, unsigned *status,
                          int n_sm, cudaStream_t s, cudaEvent_t *ev = nullptr);

// FP32 photon state (RT_MIXED: FP64 thermochemistry; RT_MIXED32, rates32:
// FP32 rate transcendentals and absorption coefficients, FP64 updates).
cudaError_t launch_thermo_mixed(const ThermoParams &tp, int G, bool rates32, const double *nH, double *xHII,
                                double *xHeII, double *xHeIII, double *T, float *N, float *F, float *Npre,
                                float *Fpre, int32_t *subcycles, Queue q, unsigned *status, int n_sm,
                                cudaStream_t s, cudaEvent_t *ev = nullptr);

// the kernels of one precision family for every group count (thermo_f64.cu,
// thermo_f64_sm.cu, thermo_mix.cu, thermo_mix_sm.cu, thermo_mix32.cu,
// thermo_mix32_sm.cu)
#define RTGB_THERMO_DISPATCH(NAME, P)                                                                               \
    cudaError_t NAME(const ThermoParams &tp, int G, const double *nH, double *xHII, double *xHeII, double *xHeIII, \
                     double *T, P *N, P *F, P *Npre, P *Fpre, int32_t *subcycles, Queue q, unsigned *status,     \
                     int n_sm, cudaStream_t s, cudaEvent_t *ev);
RTGB_THERMO_DISPATCH(thermo_dispatch_f64, double)
RTGB_THERMO_DISPATCH(thermo_dispatch_f64_sm, double)
RTGB_THERMO_DISPATCH(thermo_dispatch_mix, float)
RTGB_THERMO_DISPATCH(thermo_dispatch_mix_sm, float)
RTGB_THERMO_DISPATCH(thermo_dispatch_mix32, float)
RTGB_THERMO_DISPATCH(thermo_dispatch_mix32_sm, float)
#undef RTGB_THERMO_DISPATCH



cudaError_t launch_inject(int nsrc, int G, long long nc, const long long *cells,
                          const double *Lsum, double dt_over_V, double *N, cudaStream_t s);

cudaError_t launch_reduce_N(int G, long long nc, const double *N, const Partials &p,
                            cudaStream_t s);
cudaError_t launch_inject_f32(int nsrc, int G, long long nc, const long long *cells, const double *Lsum,
                              double dt_over_V, float *N, cudaStream_t s);
cudaError_t launch_reduce_N_f32(int G, long long nc, const float *N, const Partials &p, cudaStream_t s);
cudaError_t launch_convert_d2f(long long n, const double *in, float *out, cudaStream_t s);
cudaError_t launch_scale(long long n, double f, double *x, cudaStream_t s);        // x *= f
cudaError_t launch_scale_f32(long long n, double f, float *x, cudaStream_t s);
cudaError_t launch_convert_f2d(long long n, const float *in, double *out, cudaStream_t s);

// ---- adjoint (adjoint.cu) ----
// thermo_vjp: lambda' (gas lx..lT in place; photons lN_in/lF_in) of the
// state after the thermochemistry -> lambda of the state U_b before it
// (gas in place, photons to lN_out/lF_out); g_nH += dJ/dn_H.  N, F, gas:
// U_b.  sub_out (optional): attempts of the recomputation per cell.
cudaError_t launch_thermo_vjp(const ThermoParams &tp, int G, const double *nH, const double *xHII,
                              const double *xHeII, const double *xHeIII, const double *T, const double *N,
                              const double *F, double *lx, double *ly2, double *ly3, double *lT,
                              const double *lN_in, const double *lF_in, double *lN_out, double *lF_out,
                              double *g_nH, int32_t *sub_out, unsigned *status, cudaStream_t s);
// transport_vjp (GLF or HLL): lambda of the transported photons (lN1, lF1)
// -> lambda of the photons before transport (lN0, lF0); N, F: the state
// before it.
cudaError_t launch_transport_vjp(const GridDev &g, int G, int flux, double cr, double dt, const double *N,
                                 const double *F, const double *hll_table, const double *inflow,
                                 const double *lN1, const double *lF1, double *lN0, double *lF0, cudaStream_t s);
// transpose of the |F| <= c N rescaling of the transport output N, F, in
// place on lN, lF
cudaError_t launch_clamp_vjp(int G, long long nc, double cr, const double *N, const double *F, double *lN, double *lF,
                             cudaStream_t s);
// g_L[s][i] += lN[i][cells[s]] dt / V for every source s (unmerged list)
cudaError_t launch_inject_vjp(int nsrc, int G, long long nc, const long long *cells, const double *lN,
                              double dt_over_V, double *g_L, cudaStream_t s);
cudaError_t launch_count_mismatch(long long n, const int32_t *a, const int32_t *b, unsigned long long *count,
                                  cudaStream_t s);

int reduce_blocks_per_group();

// budget[G][4] cumulative: in_box, absorbed, outflow, emitted.  mode 0
// closes a step (emitted[G] = photons emitted in it, host array baked into
// the launch); mode 1 re-initialises at set_state.  Also resets the queue.
cudaError_t launch_finalize_mode(int G, int mode, const Partials &p, double V, const double *emitted,
                                 double *budget, Queue q, unsigned *status, cudaStream_t s);

void hll_table(int nf, int nmu, double *out);
void hll_speeds(double f, double mu, double *lmin, double *lmax);

}  // namespace rtgb
