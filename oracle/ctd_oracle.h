/*
 * ctd_oracle.h -- CPU oracle for the gCTD photon transport (TEST INFRASTRUCTURE).
 *
 * This header and ctd_oracle.c are a plain, slow, single-threaded restatement of
 * the method of Jia, Yan, Gu and Jiang, "Fast Monte Carlo Simulation for
 * Patient-specific CT/CBCT Imaging Dose Calculation" (arXiv:1109.3266):
 * Woodcock tracking (Sec. 2.1), interaction choice (Sec. 2.1), R/C-surface
 * angular sampling (Sec. 2.2.2, Eq. 1; Sec. 2.2.3, Eq. 2), local deposition
 * (Sec. 2.1), stratified spectrum (Sec. 2.2.5), source trajectory (Sec. 2.2.6)
 * and batches (Sec. 2.2.1).
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this code.  The product library never links or calls it,
 * and it shares no source with the product library.
 *
 * Every function exists in two precisions built from one source:
 *   *_f64 : the method in IEEE binary64 with the C library's log/sin/cos/sqrt;
 *   *_f32 : a second restatement in the paper's single precision (Sec. 2.2.7
 *           item 1), with the single-precision log and sincos defined in
 *           ctd_oracle.c, so that integer decisions (interaction type, voxel
 *           index, escape) are taken in binary32; the CPU tests compare it with
 *           *_f64 history by history under the decision margins below.
 * Integer-only helpers (Philox, allocation) have one version.
 */
#ifndef CTD_ORACLE_H
#define CTD_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Material record: the closed-form cross sections need these numbers. */
#define OR_MAX_ELEMENTS 16

typedef struct {
    double z_over_a;  /* electrons per gram / N_A (Compton, Eq. 2)                 */
    double a_mol;     /* molar mass of one formula unit, g/mol (PE and Rayleigh)   */
    double z_eff;     /* effective atomic number (PE ~ Z^4, Rayleigh ~ Z^2)         */
    double q0;        /* analytic form-factor width, 1/Angstrom; <= 0 means F^2 = 1 */
    double sq0;       /* analytic scattering-function width for the Waller-Hartree
                         Compton model, S(q)/Z = 1 - exp(-q^2/sq0^2), 1/Angstrom;
                         <= 0 means S/Z = 1 (free electrons)                      */
    /* elements of one formula unit for the independent-atom (IAA) molecular form
     * factor of Rayleigh scattering: n_el > 0 selects it for the material's Rayleigh
     * total and R surface (n_el = 0: F^2 = exp(-q^2/q0^2) and the closed-form total) */
    int n_el;
    int el_z[OR_MAX_ELEMENTS];    /* atomic numbers, 1..100 */
    double el_n[OR_MAX_ELEMENTS]; /* atoms per formula unit, > 0 */
} or_material;

enum { OR_SRC_STATIC = 0, OR_SRC_ARC = 1 };
enum { OR_MODE_FULL = 0, OR_MODE_MAX_REAL = 1 };
enum { OR_SAMPLE_SURFACE = 0, OR_SAMPLE_EXACT = 1 };
/* Compton model (Sec. 2.2.3): free-electron Klein-Nishina (Eq. 2 with S = 1) or
 * Waller-Hartree (Eq. 2 with the material's scattering function S(q)). */
enum { OR_COMPTON_KN = 0, OR_COMPTON_WH = 1 };

typedef struct {
    /* phantom: x fastest, then y, then z; centred at the origin */
    int nx, ny, nz;
    double dx, dy, dz;            /* cm */
    const uint8_t *mat;           /* material index per voxel */
    const float *rho;             /* density per voxel, g/cm^3 */
    int n_mat;
    const or_material *mats;
    /* source */
    int src_kind;                 /* OR_SRC_STATIC: from (0,0,-sad) along +z; OR_SRC_ARC: about z */
    double sad;                   /* source-to-centre distance, cm */
    double u_lo, u_hi, v_lo, v_hi;/* field at the centre plane, cm */
    int n_proj;                   /* discrete projections on the arc */
    double arc0, arc1;            /* arc start/end, radians */
    int continuous;               /* 1: angle uniform on [arc0, arc1) (Sec. 2.2.6) */
    double z0, z1;                /* arc source height at arc0 and at arc1, linear in the
                                     angle (helical trajectory; 0, 0: circular), cm      */
    /* fluence map (Sec. 2.2.4): fl_nu x fl_nv beamlets tiling the field, u fastest,
     * relative intensities fl_f (>= 0, sum > 0); fl_nu = 0: no map (uniform in solid angle) */
    int fl_nu, fl_nv;
    const double *fl_f;
    /* spectrum: bins [e_lo, e_hi] keV with relative weight w (Sec. 2.2.5) */
    int nbins;
    const double *e_lo, *e_hi, *w;
    /* physics */
    int e_min, e_max;             /* node grid e_min..e_max keV step 1; e_min is the cutoff */
    int n_zeta;                   /* surface columns in zeta */
    double majorant_scale;        /* >= 1 */
    int mode;                     /* OR_MODE_* */
    int max_real;                 /* real interactions before termination (OR_MODE_MAX_REAL) */
    int sampling;                 /* OR_SAMPLE_* (EXACT only in f64) */
    int compton;                  /* OR_COMPTON_* */
    /* run */
    uint64_t n_hist;
    int n_batches;
    uint64_t seed;
} or_problem;

/* Integer counts: one slot per outcome. */
typedef struct {
    uint64_t pe, compton, rayleigh, fictitious;
    uint64_t escaped, missed, cutoff, terminated, aborted;
    uint64_t steps;
    double e_emitted, e_escaped, e_deposited;  /* keV */
} or_counts;

/* Philox4x32-10, Salmon et al. (SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform(uint32_t x);

/* closed forms, cm^2/g, E in keV */
double or_sigma_kn(double e_kev);                  /* cm^2 per electron */
double or_mu_pe(const or_material *m, double e_kev);
double or_mu_compton(const or_material *m, double e_kev);
double or_mu_rayleigh(const or_material *m, double e_kev);
/* Waller-Hartree: pi r0^2 times the composite Simpson integral over mu in
 * [-1, 1] (20000 intervals) of (E'/E)^2 (E'/E + E/E' - sin^2 theta) S(q)/Z,
 * cm^2 per electron; sq0 <= 0 integrates Klein-Nishina alone */
double or_sigma_wh(double e_kev, double sq0);
double or_mu_compton_wh(const or_material *m, double e_kev);
/* Independent-atom molecular form factor (Sec. 2.2.2, Eq. 1), a screened
 * hydrogenic atom per element: F_Z(x) = Z / (1 + (2 pi a_Z x)^2)^2 with the
 * Thomas-Fermi radius a_Z = 0.8853 a0 Z^(-1/3), x = sin(theta/2)/lambda in
 * 1/Angstrom; F^2_mol(x) = sum_i n_i F_Zi(x)^2.  Arguments: x^2. */
double or_ff_atom2(int z, double x2);
double or_ff_mol2(const or_material *m, double x2);
/* Rayleigh total per formula unit in cm^2 with the IAA form factor: pi r0^2 times
 * the composite Simpson integral over mu in [-1, 1] (20000 intervals) of
 * (1 + mu^2) F^2_mol(x), x^2 = k^2 (1 - mu) / 2, k = E / hc */
double or_sigma_rayleigh_iaa(const or_material *m, double e_kev);
double or_mu_rayleigh_iaa(const or_material *m, double e_kev);

/* integer allocation of n histories to bins by largest remainder */
int or_allocate(uint64_t n, int nbins, const double *w, uint64_t *out);

/* single-precision elementary functions of the f32 method */
float or_log_f32(float u);
void or_sincos_turns_f32(float t, float *c, float *s);
void or_eval_log_f32(const float *u, float *out, size_t n);
void or_eval_sincos_f32(const float *t, float *c, float *s, size_t n);
void or_eval_uniform_f32(const uint32_t *x, float *out, size_t n);   /* or_uniform in binary32, n words */

/* problem set-up (tables and surfaces) and transport of a history range.
 * Parity unpinned for the full multiple-scatter dose in heterogeneous phantoms:
 * nothing independent of this code gives it (no EGSnrc or PENELOPE data here).
 * The transport rests on its pinned parts (cross sections, surfaces, sampling,
 * allocation, Philox), on closed forms in slabs and pencil beams with one or two
 * real interactions, on energy conservation, and on the binary64 and binary32
 * runs agreeing history by history under the decision margins below. */
typedef struct or_setup or_setup;
or_setup *or_setup_create_f64(const or_problem *p);
or_setup *or_setup_create_f32(const or_problem *p);
void or_setup_destroy(or_setup *s);
int or_transport_f64(const or_setup *s, uint64_t h0, uint64_t h1, double *edep, or_counts *c);
int or_transport_f32(const or_setup *s, uint64_t h0, uint64_t h1, double *edep, or_counts *c);

/* Per-history records with decision margins (the primary-only comparison of
 * the interaction choice, Sec. 2.1, against a single-precision run).
 *
 * Every integer decision of a history -- the source's acceptance test, the
 * miss test at the box, escape, the voxel a flight ends in, the interaction
 * type and the Compton cutoff -- compares two numbers.  The binary64 run logs,
 * for each decision, the gap between them divided by a bound on how far a
 * binary32 evaluation of the same numbers can be off (a few units of 2^-24 of
 * the quantities involved; the bounds are stated in ctd_oracle_transport.inc).
 * `margin` is the smallest such ratio over the decisions that change the
 * history's path; `margin_loc` also takes the voxel boundaries that change only
 * where a deposit lands.  A history with margin >= 1 must take every decision
 * the same way in binary32; one below 1 may legitimately differ.  The bounds
 * hold up to the first real interaction (all of a primary-only history); after
 * a scatter the direction's error is not bounded here.  The binary32 run
 * leaves both margins at +inf. */
enum { OR_END_PE = 0, OR_END_CUTOFF = 1, OR_END_ESCAPED = 2, OR_END_MISSED = 3, OR_END_TERMINATED = 4,
       OR_END_ABORTED = 5 };
enum { OR_MARGIN_NONE = 0, OR_MARGIN_ACCEPT = 1, OR_MARGIN_ENTRY = 2, OR_MARGIN_ESCAPE = 3,
       OR_MARGIN_BOUNDARY = 4, OR_MARGIN_TYPE = 5, OR_MARGIN_CUTOFF = 6 };
typedef struct {
    int32_t end;          /* OR_END_*                                                        */
    int32_t last_type;    /* last real interaction: 0 photoelectric, 1 Compton, 2 Rayleigh, -1 none */
    uint32_t steps;       /* Woodcock steps taken                                            */
    uint32_t idx;         /* voxel of the last real interaction (0xffffffff: none)            */
    double e_end;         /* keV deposited by the event that ended the history (0 if none)   */
    double margin;        /* see above                                                       */
    double margin_loc;
    int32_t margin_kind;  /* OR_MARGIN_* of `margin`                                         */
    int32_t pad;
} or_track;
int or_track_f64(const or_setup *s, uint64_t h0, uint64_t h1, or_track *out);
int or_track_f32(const or_setup *s, uint64_t h0, uint64_t h1, or_track *out);

/* inspection of the set-up (node values as stored; f32 values widened) */
int or_setup_sizes(const or_setup *s, int *n_e, int *n_zeta, int *n_mat);
void or_setup_tables(const or_setup *s, double *mu_cum /* n_mat*n_e*3 */, double *mu_max /* n_e */);
void or_setup_surfaces(const or_setup *s, double *c_surf /* n_c*n_e*n_zeta, n_c = 1 (KN) or n_mat (WH) */,
                       double *r_surf /* n_mat*n_e*n_zeta */);

/* the surfaces on their own (Sec. 2.2.2 and 2.2.3), binary64 */
void or_build_kn_surface(int e_min, int n_e, int n_zeta, double *out);
void or_build_rayleigh_surface(double q0, int e_min, int n_e, int n_zeta, double *out);
void or_build_rayleigh_iaa_surface(const or_material *m, int e_min, int n_e, int n_zeta, double *out);
void or_build_wh_surface(double sq0, int e_min, int n_e, int n_zeta, double *out);

/* angular samplers for the sampler validation of Figs. 3-4:
 * kind 0 = Compton (the set-up's model; Waller-Hartree reads the material's
 * scattering function), 1 = Rayleigh;
 * surface samplers read the set-up's surfaces at E; exact samplers use rejection. */
int or_sample_mu_f64(const or_setup *s, int kind, int material, double e_kev, int exact,
                     uint64_t seed, uint64_t n, double *out);
int or_sample_mu_f32(const or_setup *s, int kind, int material, double e_kev,
                     uint64_t seed, uint64_t n, double *out);

/* Fluence map (Sec. 2.2.4).  Alias table of n intensities f (Walker's method in
 * Vose's construction): beamlet I is drawn from a 32-bit word x and a second
 * word y as k = floor(x n / 2^32), I = k if y < thr[k] else alias[k].
 * Returns 0, or -1 if the intensities are unusable. */
int or_alias_build(int n, const double *f, uint32_t *thr, int32_t *alias);
/* Beamlet counts of n particles drawn from the alias table with the source's
 * random numbers (particle i: Philox block (i, 1, stream 1) under seed). */
void or_alias_counts(int n_f, const uint32_t *thr, const int32_t *alias, uint64_t n, uint64_t seed,
                     uint64_t *counts);
/* Beamlet counts of n particles from the paper's Metropolis-Hastings chain
 * (Algorithm A1) started at beamlet i0: trial J uniform, kept if zeta < f_J /
 * f_last (particle i: Philox block (i, 0, stream 4) under seed). */
void or_mh_counts(int n_f, const double *f, int i0, uint64_t n, uint64_t seed, uint64_t *counts);
/* The same with one chain per GPU thread, as the paper runs A1: chain c of `chains`
 * takes particles [n c / chains, n (c + 1) / chains) (the first n mod chains
 * chains one more), each starting at i0; counts summed over the chains. */
void or_mh_chains(int n_f, const double *f, int i0, uint64_t n, uint64_t seed, uint64_t chains, uint64_t *counts);

/* the direction rotation on its own, for invariant checks */
void or_rotate_f64(double *u, double mu, double t_phi);
void or_rotate_f32(float *u, float mu, float t_phi);

#ifdef __cplusplus
}
#endif
#endif
