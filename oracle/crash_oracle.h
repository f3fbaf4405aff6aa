/*
 * crash_oracle.h -- plain sequential FP64 CPU oracle of one CRASH2-style
 * Monte-Carlo radiative-transfer step (emission, cell-by-cell transport with
 * attenuation and deposition, per-cell ionisation network and temperature).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library) never calls it and shares no code with it.
 *
 * Paper sections followed: Sec. 2 (packet emission, Eq. 1 attenuation,
 * species split, ionisation network, continuous processes, termination,
 * diffuse recombination field), Sec. 3 (re-emission of the diffuse field)
 * and Sec. 3.2 (N_p/N_t packets per source per step, sub-sampled chemistry).
 */
#ifndef CRASH_ORACLE_H
#define CRASH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* field ids for oracle_read_fields / oracle_write_fields */
enum {
  OR_F_XHII = 0, OR_F_XHEII = 1, OR_F_XHEIII = 2, OR_F_T = 3,   /* f64 per cell */
  OR_F_DEP_HI = 4, OR_F_DEP_HEI = 5, OR_F_DEP_HEII = 6, OR_F_DEP_E = 7, /* i64 per cell */
  OR_F_BUDGET = 8,                                              /* i64[8] */
  OR_F_NH = 9,                                                  /* f64 per cell (read only) */
  /* f64 per cell (r/w): photons of recombinations to the ground state of
     H I, He I and He II waiting for re-emission (diffuse field on) */
  OR_F_REC_HI = 11, OR_F_REC_HEI = 12, OR_F_REC_HEII = 13
};

typedef struct {
  int nx, ny, nz;
  double box_cm;                 /* length of the x edge; cells are cubes of box_cm/nx */
  const float* n_H;              /* nx*ny*nz, cm^-3, x fastest; NULL => n_H0 */
  double n_H0;
  double he_over_h;              /* n_He / n_H by number; 0 => pure hydrogen */
  const double *x_HII, *x_HeII, *x_HeIII, *T;   /* NULL => uniform values below */
  double x_HII0, x_HeII0, x_HeIII0, T0;
  int isothermal, caseB;
  double z_compton;              /* < 0: Compton term off */
  uint64_t seed;
  double f_rec;                  /* > 0: diffuse recombination radiation with this
                                    re-emission threshold (Sec. 2); 0: off */
  int coupling;                  /* transport -> chemistry: 0 = photo-ionisation rate per
                                    frozen absorber (default); 1 = photon-conserving: the
                                    step's absorbed photons ionise at a constant rate, at
                                    most the atoms present; the rest are lost */
  int periodic;                  /* 1: periodic box (Sec. 2): a packet leaving a face
                                    re-enters at the opposite one and stops after the
                                    distance light travels in the step, c dt */
  double uv_rate[3];             /* uniform background (Sec. 2 "background field", a
                                    reading): photo-ionisations per atom of H I, He I,
                                    He II and s, the same in every cell and not
                                    attenuated; 0 = off */
  double uv_heat_eV[3];          /* energy each such photo-ionisation leaves as heat, eV */
} or_grid_desc;

typedef struct or_ctx or_ctx;

/* --- context API (same shape as the CUDA library's C ABI) --- */
or_ctx* oracle_init_grid(const or_grid_desc* d);
int oracle_add_sources(or_ctx* c, int n_src, const double* pos, const double* ndot,
                       int n_bins, const double* bin_eV, const double* bin_frac);
int oracle_set_options(or_ctx* c, int chemistry, uint32_t pkt_begin, uint32_t pkt_end,
                       double chem_eps, int chem_max_sub, int cool_mask);
int oracle_step(or_ctx* c, double dt_s, uint64_t packets_per_step);
int oracle_read_fields(or_ctx* c, int field_id, void* out);
int oracle_write_fields(or_ctx* c, int field_id, const void* in);
int oracle_set_step_index(or_ctx* c, uint64_t step);
/* Timing sample of the per-cell update (CPU baseline only; 1 and 1.0 are
   the full step): update only the cells whose index is a multiple of
   chem_stride, with every deposit multiplied by dep_scale (the deposits a
   full step would make when only a window of packet ids was traced). */
int oracle_set_chem_sample(or_ctx* c, uint32_t chem_stride, double dep_scale);
/* exchange of a step split over processes (the library's crash_write_deposits
   and crash_chemistry): deposits int64[cells][4], then the per-cell update
   of the last step, run without chemistry, with that step's dt */
int oracle_write_deposits(or_ctx* c, const int64_t* in);
int oracle_chemistry(or_ctx* c, double dt_s);
void oracle_free(or_ctx* c);
const char* oracle_last_error(or_ctx* c);

/* --- building blocks exposed for pinning tests --- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_exp_neg(double tau);
int or_direction(uint64_t seed, uint32_t step, uint32_t src, uint32_t pkt, double d[3]);
void or_cross_sections(int n_bins, const double* E_eV, double* sigma /* 3*n_bins */);
/* trace one packet of n_bins contents from pos along dir through the frozen
   absorbers of c; writes deposits into c's counters; returns crossings;
   escaped content is added to *escaped; optional per-segment log. */
int64_t or_trace_packet(or_ctx* c, const double pos[3], const double dir[3],
                        int64_t* content, int64_t* escaped, int64_t* absorbed,
                        int max_log, int64_t* log_cell, double* log_len, int* n_log);
int or_freeze_absorbers(or_ctx* c);   /* absorbers from the current state; zero deposits */
/* start of the re-emission packet of cell `cell` at step `step` (grid units,
   inside the cell) and its direction; returns the direction attempts used */
int or_rec_start(uint64_t seed, uint32_t step, int64_t cell, int nx, int ny, double pos[3],
                 double dir[3]);

/* one cell of the ionisation network + temperature over dt (Sec. 2, Sec. 3.2) */
typedef struct {
  double nH, nHe;
  double xHII, xHeII, xHeIII, T;
  double G_HI, G_HeI, G_HeII;       /* photoionisation rate per absorber, s^-1 */
  double heat_per_ion;              /* mean photo-electron energy per absorbed photon, erg */
  double S_HI, S_HeI, S_HeII;       /* constant photo-ionisations per atom of the element,
                                       s^-1 (photon-conserving coupling); in a sub-step each
                                       ionises at most the atoms of its species present */
  double heat_rate;                 /* constant photo-heating, erg cm^-3 s^-1 */
  double U_HI, U_HeI, U_HeII;       /* uniform background photo-ionisation rate per atom of
                                       the species, s^-1 (added to G_*) */
  double Ue_HI, Ue_HeI, Ue_HeII;    /* heat per such photo-ionisation, erg */
  int isothermal, caseB;
  double T_cmb;                     /* <= 0: Compton off */
  double eps;                       /* relative change allowed per sub-step */
  int max_sub;
  int cool_mask;                    /* OR_C_* bits of processes switched on */
  int count_rec;                    /* 1: count recombinations to the ground state */
  double rec[3];                    /* out (added to): such recombinations per cm^3 into
                                       H I, He I, He II over dt */
} or_chem_t;

enum {
  OR_C_COLL_EXC = 1, OR_C_COLL_ION = 2, OR_C_RECOMB = 4, OR_C_BREMS = 8,
  OR_C_COMPTON = 16, OR_C_DIELEC = 32, OR_C_ALL = 63
};
int or_chem_cell(or_chem_t* c, double dt);

/* rate coefficients at T: out[0..6] = alpha_HII, alpha_HeII, alpha_HeIII,
   alpha_dielectronic, beta_HI, beta_HeI, beta_HeII (cm^3 s^-1);
   out[7..] = cooling coefficients (erg cm^3 s^-1): exc_HI, exc_HeII,
   ion_HI, ion_HeI, ion_HeII, rec_HII, rec_HeII, rec_HeIII, diel, brems(gff*sqrt(T)*1.42e-27) */
void or_rates(double T, int caseB, double out[17]);
double or_compton_coef(double T_cmb);   /* erg s^-1 K^-1 per electron */

#ifdef __cplusplus
}
#endif
#endif
