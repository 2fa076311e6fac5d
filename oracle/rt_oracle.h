/*
 * Oracle interface (test infrastructure only; see rt_oracle.c).
 * Plain FP64 CPU statement of one RT step of Rosdahl et al. 2013.
 */
#ifndef RT_ORACLE_H
#define RT_ORACLE_H
#include <stdint.h>

#define ORACLE_MAXG 8

enum { ORACLE_GLF = 0, ORACLE_HLL = 1 };
enum { ORACLE_BC_OUTFLOW = 0, ORACLE_BC_REFLECT = 1, ORACLE_BC_PERIODIC = 2, ORACLE_BC_INFLOW = 3 };
enum { ORACLE_OK = 0, ORACLE_EINVAL = -1, ORACLE_ESUBCYCLE = -3 };

/* indices into the rate arrays filled by oracle_rates */
enum {
    R_BETA_HI, R_BETA_HEI, R_BETA_HEII,
    R_ALPHA_HII, R_ALPHA_HEII, R_ALPHA_HEIII,
    R_ZETA_HI, R_ZETA_HEI, R_ZETA_HEII,
    R_ETA_HII, R_ETA_HEII, R_ETA_HEIII,
    R_PSI_HI, R_PSI_HEII,
    R_THETA, R_VARPI, R_OMEGA_HEII,
    R_COUNT
};

typedef struct {
    int nx, ny, nz;
    double dx;              /* cell width [cm] */
    int bc[6];              /* -x,+x,-y,+y,-z,+z */
    int G;                  /* photon groups */
    double cr;              /* reduced light speed [cm/s] */
    const double *sigN;     /* [G][3] cm^2, species HI, HeI, HeII */
    const double *sigE;     /* [G][3] cm^2 */
    const double *egy;      /* [G] erg */
    double X;               /* hydrogen mass fraction */
    int isothermal;
    int otsa;
    int flux;               /* ORACLE_GLF / ORACLE_HLL */
    double a_exp;           /* expansion factor for Compton */
    int max_subcycles;
    const double *hll_table;/* [nf][nmu][2] lambda_min, lambda_max / c */
    int hll_nf, hll_nmu;
    int nthreads;           /* OpenMP threads over cells (<=1: serial) */
    int skip_thermo;        /* transport-only tests */
    int smooth;             /* smoothed RT, Sec. 3.4 */
    int rec_group[3];       /* without OTSA: group that HII, HeII, HeIII
                               recombinations emit into (-1: none) */
    const double *inflow;   /* [6][G][4] ghost (N, Fx, Fy, Fz) of inflow faces, or NULL (0) */
} oracle_cfg;

void oracle_rates(double T, double a_exp, int case_b, double *r, double *dr);
double oracle_chi(double f);
void oracle_eddington(double c, double N, const double F[3], double D[9],
                      double *f_out, double n_out[3]);
void oracle_hll_lookup(const double *tab, int nf, int nmu, double f, double mu,
                       double *lmin, double *lmax);
int oracle_thermo_cell(const oracle_cfg *cfg, double dt_rt, double nH, double *s,
                       double *N, double *F, const double *Ndot, const double *Fdot,
                       int fixed_photons, int *attempts_out, double *absorbed_out,
                       double *margin_out);
double oracle_courant_dt(double cfl, double dx, double cr);
int oracle_step(const oracle_cfg *cfg, double dt, const double *nH, double *xHII,
                double *xHeII, double *xHeIII, double *T, double *N, double *F,
                int nsrc, const int32_t *src_ijk, const double *src_L,
                double *budget, int32_t *subcycles, double *margins);
#endif
