/*
 * ctd.h -- C ABI of the GB300 photon Monte Carlo dose engine (method of Jia,
 * Yan, Gu, Jiang, "Fast Monte Carlo Simulation for Patient-specific CT/CBCT
 * Imaging Dose Calculation", arXiv:1109.3266).
 *
 * Conventions for every call:
 *   - the return value is a ctd_status; on failure ctd_last_error() returns a
 *     message for the calling thread; no call aborts the process;
 *   - pointers are host pointers unless the name ends in _dev; the caller owns
 *     every buffer it passes and the library copies what it keeps;
 *   - voxel arrays are x fastest, then y, then z (index x + nx*(y + ny*z));
 *   - units: cm, g/cm^3, keV, radians; dose in Gy per source history;
 *   - a context is used by one host thread at a time;
 *   - all work runs on the context's CUDA stream; calls that return results to
 *     the host synchronise that stream.
 */
#ifndef CTD_H
#define CTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CTD_ABI_VERSION 9

/* largest number of elements of one material's formula unit (ctd_set_material_elements) */
#define CTD_MAX_ELEMENTS 16

typedef enum {
    CTD_OK = 0,
    CTD_EINVAL = 1,       /* an argument is out of range or inconsistent   */
    CTD_ENOMEM = 2,       /* device or host allocation failed              */
    CTD_ECUDA = 3,        /* a CUDA runtime call failed                    */
    CTD_EBUSY = 4,        /* the object is in use by a running request     */
    CTD_ETIMEOUT = 5,     /* a bounded wait ran out                        */
    CTD_ECANCELLED = 6,   /* the request was cancelled                     */
    CTD_ENOTFOUND = 7     /* unknown handle                                */
} ctd_status;

typedef struct ctd_ctx ctd_ctx;
typedef int32_t ctd_phantom;

/* Context options.  Zero fields take defaults. */
typedef struct {
    int device;               /* CUDA device ordinal                                  */
    void *stream;             /* cudaStream_t to launch on; NULL: the context makes one */
    int blocks_per_sm;        /* transport grid = SMs x blocks_per_sm (default 4)     */
    int threads_per_block;    /* multiple of 32, <= 256 (default 256)                */
    int chunk;                /* histories a warp claims at a time (default 256)      */
    int flight_cap;           /* Woodcock flights a lane takes in a row, stopping early at a
                                 real interaction, before its warp moves on (default 4) */
    int multi_blocks_per_sm;  /* grid of multi-request launches (batched, served; default 3) */
    int serve_max_active;     /* served requests running at once (default 64)         */
    double serve_round_histories; /* requests are admitted first in, first out while one
                                 batch of every running request stays within this many
                                 histories (default 1e8); one request always runs     */
    double serve_reserve_bytes; /* served form: a request is admitted only while the device's
                                 free memory exceeds what its buffers need by this much
                                 (default 1 GiB)                                        */
    int shared_launch;        /* batched and served forms: 0 (default) runs each request's
                                 batches as its own chain of single-request launches on
                                 its own stream, so that one request's tail overlaps the
                                 next one's launch; 1 runs one multi-request launch per
                                 batch shared by all requests                          */
    int l2_persist;           /* plain-form transport launches mark the phantom's tally (1)
                                 or its packed voxel words (2) as persisting in L2 (an
                                 access-policy window over it, with the context's
                                 persisting-L2 limit raised to its size, at most the
                                 device's maximum, while the context lives and put back
                                 by ctd_destroy); -1 or 0 (the default): neither         */
    int plain_overlap;        /* ctd_run: 1 alternates the batches between the context's stream
                                 and a second stream of its own, each with its own tally,
                                 so that one batch's launch starts while the previous one's
                                 last blocks drain (folds stay in batch order); its launches
                                 then overlap, so each one's event-timed duration includes
                                 its neighbours'.  0 (default) or -1: every batch on the
                                 context's stream                                        */
    int batch_lanes;          /* batched form with request chains: the streams the chains
                                 share, chain k (requests largest first) on stream
                                 k mod batch_lanes, so that at most this many requests run
                                 at once (1..64; 0: 64)                                  */
} ctd_options;

/* Material: the numbers the closed-form cross sections use (Sec. 2.1).
 *   z_over_a : electrons per gram / Avogadro (Compton: N_A (Z/A) sigma_KN)
 *   a_mol    : g/mol of one formula unit (photoelectric 1e-2 Z^4/E_MeV^3 microbarn,
 *              Rayleigh 1.565e-5 Z^2/E_MeV^2 barn, both per formula unit)
 *   z_eff    : effective atomic number
 *   q0       : Rayleigh form-factor width F^2 ~ exp(-q^2/q0^2), 1/Angstrom; <= 0: F^2 = 1
 *   sq0      : scattering-function width of the Waller-Hartree Compton model,
 *              S(q)/Z = 1 - exp(-q^2/sq0^2), 1/Angstrom; <= 0: S/Z = 1 (free electrons).
 * q^2 = 2 k^2 (1 - cos theta) with k = E/hc, for both. */
typedef struct {
    double z_over_a;
    double a_mol;
    double z_eff;
    double q0;
    double sq0;
} ctd_material;

typedef enum { CTD_SRC_STATIC = 0, CTD_SRC_ARC = 1 } ctd_source_kind;

/* Source (Sec. 2.2.6).  STATIC: point at (0, 0, -sad) aimed along +z, field u
 * along x and v along y.  ARC: point at sad (sin b, cos b, 0) aimed at the
 * origin, u lateral in the xy-plane, v along z; b = arc0 + (arc1-arc0) k/n_proj
 * for a uniform integer k < n_proj, or b uniform on [arc0, arc1) if continuous.
 * The field [u_lo,u_hi] x [v_lo,v_hi] is given in cm at the plane through the
 * origin; directions are uniform in solid angle over it. */
typedef struct {
    int kind;
    double sad_cm;
    double u_lo_cm, u_hi_cm, v_lo_cm, v_hi_cm;
    int n_proj;
    double arc0_rad, arc1_rad;
    int continuous;
    double z0_cm, z1_cm;  /* ARC: source height at arc0 and at arc1, linear in the angle,
                             the field plane moving with it (helical CT); 0, 0: circle */
} ctd_source;

typedef enum { CTD_MODE_FULL = 0, CTD_MODE_MAX_REAL = 1 } ctd_mode;

/* Physics options.  Attenuation data are linear interpolation between the
 * closed forms at integer-keV nodes e_min..e_max (Sec. 2.2.7 item 3); e_min is
 * also the absorption energy (Sec. 3.1).  n_zeta columns per R/C surface row
 * (Sec. 2.2.2-2.2.3).  majorant_scale >= 1 multiplies mu_max(E) (Sec. 2.1).
 * CTD_MODE_MAX_REAL stops a photon after max_real real interactions (1 =
 * primary only), counting its remaining energy as escaped.
 * compton_model (Sec. 2.2.3): CTD_COMPTON_KN, free-electron Klein-Nishina
 * (Eq. 2 with S = 1; total in closed form, one C surface for all materials);
 * CTD_COMPTON_WH, Waller-Hartree (Eq. 2 with each material's S(q); total by
 * integration of Eq. 2 over cos theta (16-point Gauss-Legendre on 41 panels of
 * 1 - cos theta halving toward forward scattering),
 * one C surface per material). */
typedef enum { CTD_COMPTON_KN = 0, CTD_COMPTON_WH = 1 } ctd_compton_model;
typedef struct {
    int e_min_kev;
    int e_max_kev;
    int n_zeta;
    double majorant_scale;
    int mode;
    int max_real;
    int compton_model;
} ctd_physics;

/* Results of the last run of a phantom. */
typedef struct {
    uint64_t histories;
    int n_batches;
    uint64_t pe, compton, rayleigh, fictitious;   /* interactions and fictitious events */
    uint64_t escaped, missed, cutoff, terminated, aborted;  /* how histories ended       */
    uint64_t steps;                               /* Woodcock steps                        */
    double e_emitted_kev, e_escaped_kev, e_deposited_kev;
    double avg_rsd;          /* mean s/D over D > 0.1 D_max, rho >= 0.1 g/cm^3            */
    double paper_sigma_bar;  /* mean s/D_max over D > 0.2 D_max (Sec. 3.1)               */
    double d_max;            /* Gy per history                                            */
    double t_total_s;        /* wall time of the run call                                 */
    double t_transport_s;    /* device time of the transport kernels (CUDA events)        */
    int transport_launches;
} ctd_run_stats;

/* Thread-local message of the last failed call on this thread. */
const char *ctd_last_error(void);
int ctd_abi_version(void);

/* Context on one GPU.  opt may be NULL.  The context owns the stream it makes;
 * a stream passed in opt->stream stays the caller's. */
int ctd_create(ctd_ctx **out, const ctd_options *opt);
int ctd_destroy(ctd_ctx *ctx);

/* Voxel phantom (Sec. 2.2.1): nx*ny*nz voxels of dx*dy*dz cm centred at the
 * origin; mat[v] < n_mat indexes mats; density[v] is 0 or in [2^-18, 2^13)
 * g/cm^3 (the device keeps each voxel's material and density in one 32-bit word,
 * exact over that range; other values give CTD_EINVAL).  Host arrays;
 * the library copies them to the device and keeps them resident until
 * ctd_destroy_phantom.  Default physics: nodes 1..150 keV, n_zeta 1024, scale 1,
 * full transport.  Fewer than 2^32 voxels (CTD_EINVAL otherwise). */
int ctd_create_phantom(ctd_ctx *ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                       const uint8_t *mat, const float *density, int n_mat, const ctd_material *mats,
                       ctd_phantom *out);
int ctd_destroy_phantom(ctd_ctx *ctx, ctd_phantom ph);
int ctd_set_physics(ctd_ctx *ctx, ctd_phantom ph, const ctd_physics *phys);

/* Independent-atom (IAA) molecular form factor for Rayleigh scattering in
 * material `material` of phantom ph (Sec. 2.2.2, Eq. 1).  The paper takes F^2
 * from tables; the reading here: each element is a screened hydrogenic atom,
 * F_Z(x) = Z / (1 + (2 pi a_Z x)^2)^2 with the Thomas-Fermi radius
 * a_Z = 0.88534138 a0 Z^(-1/3) (a0 = 0.529177210903 Angstrom) and
 * x = sin(theta/2)/lambda, and a formula unit's F^2 is sum_i count[i] F_Z[i]^2
 * (independent atoms, no interference).  With n_el > 0 the material's Rayleigh
 * total becomes pi r0^2 times the integral over mu of (1 + mu^2) F^2 (composite
 * Gauss-Legendre as for the Waller-Hartree total), divided by a_mol for cm^2/g, and its R surface is
 * built from the same density; n_el = 0 restores F^2 = exp(-q^2/q0^2) and the
 * closed-form total.  z: n_el atomic numbers in 1..100; count: atoms per formula
 * unit, finite and > 0; both read during the call.  1 <= n_el <= CTD_MAX_ELEMENTS
 * or 0.  Errors: CTD_ENOTFOUND (phantom), CTD_EINVAL (index or values),
 * CTD_EBUSY (phantom in use by a served request). */
int ctd_set_material_elements(ctd_ctx *ctx, ctd_phantom ph, int material, int n_el, const int *z,
                              const double *count);
int ctd_set_source(ctd_ctx *ctx, ctd_phantom ph, const ctd_source *src);

/* Fluence map (Sec. 2.2.4): n_u x n_v beamlets tiling the source's field
 * rectangle at the centre plane (u fastest; f[iv * n_u + iu]) with relative
 * intensities f >= 0 of positive sum.  A source photon then comes from beamlet I
 * with probability f_I / sum f, at a point uniform inside it, instead of
 * uniformly in solid angle over the field.  The beamlet is drawn from a Walker
 * alias table built on the host in binary64 (Vose's construction; thresholds
 * floor(p 2^32) as 32-bit integers): Philox block (h, 1, stream 1) gives the
 * column k = floor(x n / 2^32), the beamlet k if y < thr[k] else alias[k], and
 * the offsets z, w inside it.  n_u = 0 removes the map.  At most 2^24 beamlets
 * and 65535 per row.
 * The host array is copied. */
int ctd_set_fluence(ctd_ctx *ctx, ctd_phantom ph, int n_u, int n_v, const double *f);
/* The alias table of the phantom's fluence map: *n beamlets, thr[n], alias[n]
 * (either pointer may be NULL; *n = 0 without a map). */
int ctd_get_fluence_table(ctd_ctx *ctx, ctd_phantom ph, int *n, uint32_t *thr, int32_t *alias);

/* The paper's Metropolis-Hastings beamlet sampler (Sec. 2.2.4, Algorithm A1) on
 * the device, as the paper runs it: `chains` independent chains, one per GPU
 * thread.  Chain c takes particles [floor(n/chains) c + min(c, n mod chains), ...)
 * of n (the first n mod chains chains one more) and starts at beamlet i0;
 * particle i draws a trial beamlet J = floor(x n_f / 2^32) and zeta =
 * (2 (y >> 9) + 1) 2^-24 from the words x, y of Philox block (i, 0, stream 4)
 * under seed, and moves to J if zeta < f_J / f_last (binary64), else stays.
 * counts[n_f] (host) receives how often each beamlet was visited.  The transport
 * draws beamlets from the alias table instead (ctd_set_fluence): a chain makes a
 * photon's beamlet depend on the particles before it in its thread.  1 <= n_f <=
 * 2^24 intensities f >= 0 (host), 0 <= i0 < n_f, 1 <= chains <= 2^32, else
 * CTD_EINVAL.  Allocates device memory for the call. */
int ctd_mh_beamlets(ctd_ctx *ctx, int n_f, const double *f, int i0, uint64_t n, uint64_t seed, uint64_t chains,
                    uint64_t *counts);

/* Spectrum (Sec. 2.2.5): nbins intervals [e_lo[j], e_hi[j]] keV (e_lo == e_hi
 * is a line) with weights w[j] >= 0, sum > 0, inside [e_min, e_max] of the
 * physics.  Each batch's histories are split over the bins by largest
 * remainder and run bin by bin with E uniform inside the bin. */
int ctd_set_spectrum(ctd_ctx *ctx, ctd_phantom ph, const double *e_lo, const double *e_hi,
                     const double *w, int nbins);

/* Helper: a synthetic tube spectrum for ctd_set_spectrum, Kramers' thick-target
 * law (kvp - E)/E on 1 keV bins [j, j+1) for j = e_min .. kvp-1, evaluated at
 * the bin middle and filtered by mm_al millimetres of aluminium with the mass
 * attenuation fit 26300/E^3 + 0.15 cm^2/g (E in keV) at 2.699 g/cm^3.  Writes
 * *nbins = kvp - e_min entries to e_lo, e_hi and w when they are non-NULL (call
 * once with NULL arrays for the count).  Host only; needs no context or GPU.
 * 1 <= e_min < kvp <= 100000, mm_al >= 0, else CTD_EINVAL. */
int ctd_spectrum_kramers(int kvp, double mm_al, int e_min, double *e_lo, double *e_hi, double *w, int *nbins);

/* Host physics of one material, as the library builds it for a phantom (host
 * only; needs no context or GPU).  Elements (n_el > 0, z, count) select the
 * independent-atom Rayleigh form factor as in ctd_set_material_elements; n_el = 0
 * the analytic one.  Node energies E_j = e_min_kev + j, j = 0 .. e_max_kev - e_min_kev.
 *
 * ctd_material_columns: the binary64 node-table columns out[3 j + c] (cm^2/g) =
 * photoelectric, + Compton (compton_model), + Rayleigh at E_j (Sec. 2.1); the
 * device holds them rounded to binary32.
 *
 * ctd_angular_surface: the binary64 inverse-CDF rows out[j n_zeta + i], mu at
 * zeta = i / (n_zeta - 1) and E_j (Sec. 2.2.2): kind 0 the Klein-Nishina C
 * surface (Eq. 2 with S = 1), 1 the material's R surface (Eq. 1), 2 its
 * Waller-Hartree C surface (Eq. 2 with S of width mat->sq0); the device holds
 * them rounded to binary32.
 *
 * Arrays are the caller's; out holds 3 n_e or n_e n_zeta doubles.  Errors:
 * CTD_EINVAL (null pointers, a bad node grid, n_zeta outside 2..2^20, an unknown
 * model or kind, element values as in ctd_set_material_elements). */
int ctd_material_columns(const ctd_material *mat, int n_el, const int *z, const double *count, int e_min_kev,
                         int e_max_kev, int compton_model, double *out);
int ctd_angular_surface(int kind, const ctd_material *mat, int n_el, const int *z, const double *count,
                        int e_min_kev, int e_max_kev, int n_zeta, double *out);

/* Host logic of a run, as the library applies it (host only; needs no context or
 * GPU).
 *
 * ctd_allocate_histories: n histories over nbins spectrum bins of weights w >= 0
 * (not all zero) by largest remainder (Sec. 2.2.5): out[j] = floor(n w_j / W) plus
 * one for the bins with the largest fractional parts (ties to the lower bin);
 * the out[j] sum to n.  One batch of a run is allocated this way.
 *
 * ctd_alias_table: the Walker alias table of a fluence map's n beamlet
 * intensities f >= 0 (finite, not all zero; Sec. 2.2.4): thresholds thr[k] =
 * floor(p_k 2^32) and aliases alias[k] of Vose's construction, as
 * ctd_get_fluence_table returns them.
 *
 * Errors: CTD_EINVAL (null pointers, nbins or n < 1, unusable weights). */
int ctd_allocate_histories(uint64_t n, int nbins, const double *w, uint64_t *out);
int ctd_alias_table(int n, const double *f, uint32_t *thr, int32_t *alias);

/* Transport n_histories in n_batches (>= 2) batches (Sec. 2.2.1) with random
 * numbers keyed by seed; afterwards mean dose and batch uncertainty are ready
 * for ctd_get_dose_and_stddev.  Blocks until the device is done. */
int ctd_run(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_histories, uint64_t seed, int n_batches);

/* Transport only histories [h_begin, h_end) of the n_histories/n_batches
 * problem (a shard: history h gives the same track in any shard) and add their
 * energy to the phantom's deposit tally, which ctd_get_edep returns; counts
 * and energies go to the stats.  The tally and stats are cleared when
 * clear != 0. */
int ctd_run_range(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_histories, uint64_t seed, int n_batches,
                  uint64_t h_begin, uint64_t h_end, int clear);

/* Sharded run: one problem of n_histories in n_batches batches split among
 * several GPUs (Sec. 4: histories distributed among GPUs that run without
 * interfering), each rank with its own context and copy of the phantom.
 * Within every batch, rank r of W transports the local histories
 * [floor(n_b r / W), floor(n_b (r + 1) / W)) of the batch's n_b, with the same
 * random numbers any other partition gives them; the ranks then sum their
 * partial batch tallies (binary64, a collective of the caller's choice) and
 * each folds the sum, so every rank holds the same batch statistics as a
 * single-GPU ctd_run, up to the order of binary64 additions.
 *   ctd_shard_begin: start the run on phantom ph (clears its sums and counts).
 *   ctd_shard_batch: transport local histories [local_begin, local_end) of batch
 *       `batch` and add their deposits (keV) to tally_dev, nvox device doubles
 *       the caller owns (asynchronously, on the context's stream).
 *   ctd_shard_fold: fold the summed batch tally tally_dev into the statistics
 *       (Sec. 2.2.1) and leave tally_dev zeroed for the next batch (asynchronous).
 *   ctd_shard_counts: this rank's counts (10: photoelectric, Compton, Rayleigh,
 *       fictitious, escaped, missed, cutoff, terminated, aborted, steps) and
 *       energies (2: emitted, escaped keV), to be summed over the ranks.
 *   ctd_shard_finish: mean dose, standard error and the precision measures of
 *       the folded batches, with the ranks' summed counts and energies as the
 *       run's stats; ctd_get_dose_and_stddev then reads the result.
 * Errors: CTD_ENOTFOUND, CTD_EINVAL (no run begun, batch or range out of range,
 * null buffers), CTD_EBUSY. */
int ctd_shard_begin(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_histories, uint64_t seed, int n_batches);
int ctd_shard_batch(ctd_ctx *ctx, ctd_phantom ph, int batch, uint64_t local_begin, uint64_t local_end,
                    double *tally_dev);
int ctd_shard_fold(ctd_ctx *ctx, ctd_phantom ph, int batch, double *tally_dev);
int ctd_shard_counts(ctd_ctx *ctx, ctd_phantom ph, uint64_t *counts, double *energies);
int ctd_shard_finish(ctd_ctx *ctx, ctd_phantom ph, const uint64_t *counts, const double *energies);

/* Per-history records for validation (the primary-only comparison of the
 * interaction choice, Sec. 2.1, and of the source, Secs. 2.2.4-2.2.6, history
 * by history).  Runs histories [h_begin, h_end) of the n_histories/n_batches
 * problem like ctd_run_range with clear != 0 (the deposit tally and stats are
 * replaced by this range's) and writes one record per history to the host
 * array out[h_end - h_begin]:
 *   code bits 0-7: how the history ended, plus one: 1 photoelectric absorption,
 *        2 Compton cutoff (E' below e_min), 3 escaped, 4 missed the phantom,
 *        5 terminated (CTD_MODE_MAX_REAL), 6 aborted (step or trial limit);
 *   code bits 8-15: type of its last real interaction plus one (1 photoelectric,
 *        2 Compton, 3 Rayleigh; 0 none);
 *   steps: Woodcock steps taken;  idx: voxel of the last real interaction
 *        (meaningful when it has one);  e_end_kev: energy deposited by the event
 *        that ended the history (0 for escaped, missed, aborted).
 * The records come from a separate instantiation of the transport kernel that
 * also writes them; the histories, random numbers and arithmetic are those of
 * ctd_run.  At most 2^26 histories per call (CTD_EINVAL beyond); the call
 * allocates 16 bytes of device memory per history for the call's duration. */
typedef struct {
    uint32_t code;
    uint32_t steps;
    uint32_t idx;
    float e_end_kev;
} ctd_track;
int ctd_trace_range(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_histories, uint64_t seed, int n_batches,
                    uint64_t h_begin, uint64_t h_end, ctd_track *out);

/* Batched form: n_req dose calculations in one call.  Request r transports
 * n_histories[r] histories of phantoms[r] (distinct phantoms, each with its
 * source and spectrum set) with random numbers keyed by seeds[r], in n_batches
 * (>= 2) batches.  The whole call is one CUDA graph, recorded once and replayed
 * while the requests and the launch shape stay the same.  With shared_launch = 0
 * each request is its own chain of single-request launches and folds on its own
 * stream, and the device overlaps one chain's last blocks with the next chain's
 * first ones; with shared_launch = 1 batch b of every request runs in one
 * multi-request launch (each warp works on one request at a time and moves on
 * to the next when it runs out of histories; all requests on the same node
 * grid, else CTD_EINVAL), followed by one fold over every request's grids.
 * Each phantom's results are then read with ctd_get_dose_and_stddev and equal
 * those of a separate ctd_run with the same arguments (up to the order of
 * binary64 additions in the tallies); its t_transport_s is the device time of
 * the whole graph (shared_launch = 0) or of its n_batches shared launches
 * (shared_launch = 1).  Blocks until done. */
int ctd_run_batch(ctd_ctx *ctx, int n_req, const ctd_phantom *phantoms, const uint64_t *n_histories,
                  const uint64_t *seeds, int n_batches);

/* ---- Served form: continuous batching of dose requests ----
 * A request transports batches of batch_histories histories of a phantom with
 * random numbers keyed by seed until, after at least min_batches batches, its
 * avg RSD is <= rsd_target, or until n_histories_max histories have run.
 * Requests wait in a queue until admitted, first in, first out (free device
 * memory above the context's reserve, serve_reserve_bytes, fewer than
 * serve_max_active running (at most 64 with shared_launch = 0), one batch of
 * every running request within serve_round_histories).
 * With shared_launch = 0 every running request advances on its own stream,
 * independently of the others: each call of ctd_serve_step takes in the
 * batches that have finished on the GPU (a batch counts only then), retires
 * requests that reached their stop and requests cancelled, admits what fits
 * and launches the next batches (transport, fold and, from min_batches on, the
 * statistics) of running requests with nothing on the GPU.  It does not wait
 * for the GPU.  Requests go in order of the histories they still need by
 * estimate (the batches up to min_batches, then the avg RSD taken to fall as
 * 1/sqrt(n); the earliest admitted among equals).  The first in line runs on a
 * stream of the device's greatest priority, every batch before its first stop
 * test in one go (work already on the GPU runs to its end: a request that
 * becomes first in line goes out at the next launch boundary).  If its batches fill the GPU (at least 64 histories per
 * resident thread of a launch), the second in line runs beside it one slice
 * (an eighth of a batch) at a time, and only while the first one's batch on the
 * GPU may be its last; if they do not, the others run, whole batches, while
 * the histories on the GPU stay below two launches that fill it.  A request
 * submitted while others run is admitted at the next call and starts there if
 * it is first in line.  With shared_launch = 1 each call runs one round, one batch of every
 * running request in one shared launch (every request on one node grid), and
 * waits for it; a round whose launches fail counts for no request and marks
 * them CTD_REQ_FAILED.
 * A finished request's result equals ctd_run(phantom, k * batch_histories,
 * seed, k) for its k batches (up to the order of binary64 additions), alone or
 * mixed with others, and is read with ctd_get_dose_and_stddev.  A phantom
 * serves one request at a time; while it does, calls that would change it
 * return CTD_EBUSY. */
typedef enum {
    CTD_REQ_QUEUED = 0,
    CTD_REQ_RUNNING = 1,
    CTD_REQ_DONE = 2,
    CTD_REQ_CANCELLED = 3,
    CTD_REQ_FAILED = 4
} ctd_req_state;

typedef struct {
    uint64_t batch_histories;   /* histories per batch (> 0)                        */
    uint64_t n_histories_max;   /* stop after this many histories (0: no limit)      */
    double rsd_target;          /* stop once avg RSD <= this (e.g. 0.01)             */
    int min_batches;            /* batches before the first check (>= 2; 0 means 10) */
    uint64_t seed;
} ctd_request;

typedef int64_t ctd_req_id;

typedef struct {
    int state;                  /* ctd_req_state                                     */
    int batches;                /* batches finished                                  */
    uint64_t histories;         /* histories finished                                */
    double avg_rsd;             /* last statistics update (0 before min_batches)      */
    double paper_sigma_bar;
    double t_queued_s;          /* time from submission to admission (so far)        */
    double t_latency_s;         /* time from submission to retirement (so far)       */
} ctd_req_status;

int ctd_submit(ctd_ctx *ctx, ctd_phantom ph, const ctd_request *req, ctd_req_id *out);
/* One step of the served form (above); *n_active (may be NULL) is the number
 * of requests still queued or running afterwards. */
int ctd_serve_step(ctd_ctx *ctx, int *n_active);
/* Steps of the served form until one of them took in, retired, admitted or
 * launched something, nothing is queued or running, or timeout_s seconds have
 * passed (>= 0, else CTD_EINVAL); between steps in which nothing happened it
 * sleeps 20 us.  *n_active (may be NULL) as for ctd_serve_step.  A request
 * loop calls it with the time until the next arrival, so that it sees each
 * batch end within tens of microseconds without spinning. */
int ctd_serve_wait(ctd_ctx *ctx, double timeout_s, int *n_active);
int ctd_poll(ctd_ctx *ctx, ctd_req_id id, ctd_req_status *out);
/* Drive ctd_serve_step until request id has finished or timeout_s seconds have
 * passed (CTD_ETIMEOUT); out may be NULL. */
int ctd_wait(ctd_ctx *ctx, ctd_req_id id, double timeout_s, ctd_req_status *out);
/* A queued request is dropped at once, a running one at the next
 * ctd_serve_step (after its batches on the GPU, if any, have finished); either
 * ends as CTD_REQ_CANCELLED. */
int ctd_cancel(ctd_ctx *ctx, ctd_req_id id);

/* Autotuner: launch-shape search for the single-request transport kernel.
 * It times probe launches of the phantom's current problem (its source,
 * spectrum and physics; the first batch of 10 * n_probe histories with seed,
 * that is n_probe histories over every 1 keV bin) for blocks of 256 threads,
 * 3 or 4 per SM, or of 128 threads, 7 or 8 per SM; claims of {64, 256, 1024}
 * histories; flight caps of {1, 2, 4, 8} (48 shapes and the context's own),
 * each best of two.  The four fastest and the context's own shape are then timed
 * again on probes five times longer, and the fastest of those is kept in the
 * context for later runs.  Results of a run do not depend on the launch shape
 * (up to the order of binary64 additions). */
typedef struct {
    int blocks_per_sm;
    int chunk;
    int flight_cap;
    int n_tried;               /* shapes timed in the first pass */
    double histories_per_s;    /* of the chosen shape on the longer probe */
    double baseline_per_s;     /* of the shape the context had before, on the longer probe */
    int threads_per_block;
    int shared_launch;         /* ctd_autotune_batch: the launch design chosen            */
    int multi_blocks_per_sm;   /* ctd_autotune_batch: blocks per SM of shared launches     */
    int batch_lanes;           /* ctd_autotune_batch: streams of the request chains        */
} ctd_tune_result;

int ctd_autotune(ctd_ctx *ctx, ctd_phantom ph, uint64_t n_probe, uint64_t seed, ctd_tune_result *out);

/* Autotuner of the batched form (the paper has no counterpart).  It times
 * ctd_run_batch of the given requests, each with probe_fraction of its histories
 * (at least one per batch), best of two calls after one that records the graph,
 * over the shapes below; then the three fastest and the context's own shape
 * again with five times the fraction (at most all of it).  The shapes: request chains with blocks of 256 threads at 4 or 3 per SM or of 128 at 8
 * per SM; shared multi-request launches at 2, 3 or 4 blocks per SM; claims of
 * 256 or 1024 histories (how many a warp takes into its photon queue at a time);
 * flight caps of 2 or 4 (how many Woodcock flights a lane runs before its warp
 * regroups at the queue); request chains sharing 2, 4, 8 or 16 streams (256
 * threads, 4 per SM, claims of 256, flight cap 4); and the context's own shape
 * (29 in all; shared
 * shapes are skipped when the requests do not share one node grid).  The
 * fastest on the longer probe is kept in the context (shared_launch,
 * threads_per_block, blocks_per_sm, multi_blocks_per_sm, chunk, flight_cap,
 * batch_lanes) and
 * returned in out (histories_per_s on the longer probe; baseline_per_s of the
 * context's previous shape there; n_tried, the shapes of the first pass).  Results do not depend on the shape (up to the order of binary64
 * additions).  The requests' phantoms end holding the last probe's results. */
int ctd_autotune_batch(ctd_ctx *ctx, int n_req, const ctd_phantom *phantoms, const uint64_t *n_histories,
                       const uint64_t *seeds, int n_batches, double probe_fraction, ctd_tune_result *out);

/* Mean dose and its standard error (Gy per history, nvox doubles each; either
 * may be NULL) and the stats of the last ctd_run (stats may be NULL). */
int ctd_get_dose_and_stddev(ctd_ctx *ctx, ctd_phantom ph, double *dose, double *stddev, size_t nvox,
                            ctd_run_stats *stats);

/* Energy deposited per voxel (keV) summed over the last run or range runs. */
int ctd_get_edep(ctd_ctx *ctx, ctd_phantom ph, double *edep_kev, size_t nvox);

/* The binary32 tables the device uses, widened to double: mu_cum[n_mat][n_e][3]
 * (photoelectric, +Compton, +Rayleigh, cm^2/g), mu_max[n_e] (1/cm),
 * c_surf[n_c][n_e][n_zeta] (n_c = 1 under Klein-Nishina, n_mat under
 * Waller-Hartree), r_surf[n_mat][n_e][n_zeta].  Sizes via the out-params
 * (any pointer may be NULL).  Builds the tables if needed. */
int ctd_get_tables(ctd_ctx *ctx, ctd_phantom ph, int *n_e, int *n_zeta, int *n_mat, double *mu_cum,
                   double *mu_max, double *c_surf, double *r_surf);

/* Sampler validation (Figs. 3-4): n polar cosines at energy e_kev drawn on the
 * device from the C surface (kind 0; under Waller-Hartree that of material)
 * or the R surface of material (kind 1),
 * the i-th from Philox counter (i, 0, 0, 3) under seed.  out: host doubles. */
int ctd_sample_mu(ctd_ctx *ctx, ctd_phantom ph, int kind, int material, double e_kev, uint64_t seed,
                  uint64_t n, double *out);

/* Device evaluation of the transport's binary32 logarithm (fn 0: out = ln x),
 * sincos of 2 pi x (fn 1: out[2i] = cos, out[2i+1] = sin) and uniform mapping
 * of a random word (fn 2: the 32 bits of x[i] taken as the word, out = its
 * uniform in (0, 1)) for n host floats; out holds 2n (fn 1) or n host floats. */
int ctd_eval_math(ctd_ctx *ctx, int fn, const float *x, float *out, size_t n);

/* Memory-system probes for the roofline of the transport kernel.  The paper has
 * no counterpart; they measure the two memory ceilings the transport meets:
 *   kind CTD_PROBE_L2_RED (0): binary64 reductions (red.global.add.f64, the
 *        deposit instruction) of 1.0 into uniformly random slots of a buffer of
 *        n_slots doubles;
 *   kind CTD_PROBE_GATHER4 (1): gathers of 4-byte records from uniformly random
 *        slots of a buffer of n_slots floats (the Woodcock step's fetch of its
 *        voxel's packed material-and-density word);
 *   kind CTD_PROBE_VOXEL (2): gathers of one voxel's material byte and 4-byte
 *        density from two arrays, uniformly random slots of n_slots voxels (the
 *        fetch a step would make without the packed word).
 * About n_ops operations (rounded up to whole rounds of 8 per thread over
 * SMs x 8 blocks of 256 threads) run in one launch, timed with CUDA events on
 * the context's stream after one untimed launch; *ops_per_s receives the mean
 * rate of 3 timed launches.  Slots are drawn with the lowbias32 hash, so
 * buffers that fit in L2 measure L2 and larger ones HBM.  The call allocates
 * and frees its buffers (CTD_ENOMEM if they do not fit) and blocks until done.
 * 1 <= n_slots < 2^32 and 1 <= n_ops <= 2^40, else CTD_EINVAL. */
enum { CTD_PROBE_L2_RED = 0, CTD_PROBE_GATHER4 = 1, CTD_PROBE_VOXEL = 2 };
int ctd_probe_memory(ctd_ctx *ctx, int kind, uint64_t n_slots, uint64_t n_ops, double *ops_per_s);

/* Allocation-free avg RSD.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need the
 * precision measure, such as hosts whose own pool allocator owns all device
 * memory and forbids library allocations.
 * It reduces dose and stddev arrays that already live on the device (nvox
 * doubles each, Gy per history) with densities density_dev (nvox floats) to
 * the same measures ctd_run reports: result_dev[0] = avg RSD (mean s/D over
 * D > 0.1 D_max, rho >= 0.1 g/cm^3), [1] = the paper's sigma_bar, [2] = D_max,
 * written to 3 device doubles, asynchronously on stream (a cudaStream_t; NULL
 * is the legacy default stream).  No context is needed; it runs on the current
 * device.  It allocates nothing: its partial sums live in a fixed 160 KB
 * device array inside the library, which every GPU that loads the library
 * holds until exit, so nvox may not exceed 67,108,864 (CTD_EINVAL beyond).
 * Each call looks up that array's device address on the current device (so a
 * device reset between calls is harmless), except on a stream that is being
 * captured, where the address that device's previous call found is used.  All calls share
 * the array: a call overwrites every partial it reads, but calls that overlap
 * on the GPU race on it. */
int ctd_avg_rsd_noalloc(const double *dose_dev, const double *stddev_dev, const float *density_dev, size_t nvox,
                        double *result_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CTD_H */
