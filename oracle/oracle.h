/* CPU oracle of the CTU-PPM hydro step — TEST INFRASTRUCTURE ONLY.
 * Loaded by the test suite, the smoke check and the benchmark's CPU-baseline
 * leg; never by the product library. */
#ifndef HYDRO_ORACLE_H
#define HYDRO_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_OK = 0, ORACLE_EINVAL = -1, ORACLE_EBADSTATE = -4 };
enum { ORACLE_BC_OUTFLOW = 0, ORACLE_BC_REFLECT = 1, ORACLE_BC_PERIODIC = 2, ORACLE_BC_PREFILLED = 3 };

typedef struct {
  int dim;            /* 2 or 3 */
  int n[3];           /* interior zones per axis; n[2] = 1 in 2-D */
  double dx[3];       /* zone widths */
  int bc[3][2];       /* boundary kind per axis, low/high side */
  double gamma;       /* gamma-law EOS exponent (> 1) */
  double cfl;         /* Courant number used by oracle_dt */
  double grav[3];     /* constant gravitational acceleration */
  double small_dens;  /* density floor */
  double small_pres;  /* pressure floor */
  int flatten;        /* 1: CW84 flattening on; 0: off */
  int wave_speeds;    /* HLLC outer wave speeds: 0 Davis, 1 Einfeldt (Roe-averaged) */
  int grav_energy;    /* gravity energy source: 0 cell-centred momentum form, 1 mass-flux form */
} oracle_params;

/* optional copies of intermediate arrays (each 5 x grown size, or 6 x for prim) */
typedef struct {
  double* prim;           /* rho,u,v,w,p,c on the grown box */
  double* trace_m[3];     /* traced state at each zone's low face, per direction */
  double* trace_p[3];     /* traced state at each zone's high face */
  double* flux1[3];       /* first (untransversed) fluxes, face f stored at zone f */
  double* flux_final[3];  /* final fluxes */
} oracle_debug;

long long oracle_grown_size(const oracle_params* P);
int oracle_fill_ghosts(double* U, const oracle_params* P);
int oracle_dt(const double* U, const oracle_params* P, double* dt_out);
int oracle_step(const double* Uin, double* Uout, const oracle_params* P, double dt, oracle_debug* dbg);
/* method-of-lines step (SSP-RK2, PPM edges, HLLC) with nspec passive species:
 * 5 + nspec fields on the grown box */
int oracle_mol_step(const double* Uin, double* Uout, const oracle_params* P, int nspec, double dt);

void oracle_hllc(const double* qL, const double* qR, int d, double gamma, double* F);
void oracle_wave_speeds(const double* qL, const double* qR, int d, double gamma, int einfeldt, double* sl_sr);
void oracle_ppm_parabola(const double* line7, double chi, double* am_ap_a6);
double oracle_flatten(const double* p7, const double* un7, double small_pres);
double oracle_integ(const double* am_ap_a6, double sigma, int plus);
void oracle_trace_lines(const double* lines6x7, int d, const oracle_params* P, double dtdx, double dt,
                        double* qm, double* qp);
void oracle_cons_to_prim(const double* U, const oracle_params* P, double* q, int* bad);
void oracle_prim_to_cons(const double* q, double gamma, double* U);

/* counting build only (liboracle_count.so): operation tallies */
void oracle_tally_reset(void);
void oracle_tally_get(long long* out5);
void oracle_tally_stages(long long* out30);

/* exact Riemann solver for the gamma-law Euler equations */
int oracle_exact_star(const double* WL, const double* WR, double gamma, double* pstar_ustar);
int oracle_exact_sample(const double* WL, const double* WR, double gamma, const double* xi, int n, double* W_out);

#ifdef __cplusplus
}
#endif
#endif
