// ctd_internal.h -- internal declarations of the dose engine library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ctd.h"

namespace ctd {

// physical constants (CODATA 2018)
constexpr double kMec2 = 510.99895;             // electron rest energy, keV
constexpr double kR0 = 2.8179403262e-13;        // classical electron radius, cm
constexpr double kNA = 6.02214076e23;           // Avogadro, 1/mol
constexpr double kHc = 12.398419843320026;      // h c, keV Angstrom
constexpr double kPi = 3.141592653589793;
constexpr double kMicrobarn = 1.0e-30;          // cm^2
constexpr double kBarn = 1.0e-24;               // cm^2
constexpr double kPeCoef = 1.0e-2;              // photoelectric coefficient, microbarn
constexpr double kRayCoef = 1.565e-5;           // Rayleigh coefficient, barn MeV^2
constexpr double kKevToJ = 1.602176634e-16;
constexpr int kCdfIntervals = 20000;            // mu intervals of the numeric cdf
constexpr double kBohr = 0.529177210903;         // Bohr radius, Angstrom
constexpr double kThomasFermi = 0.88534138;     // Thomas-Fermi radius / (a0 Z^-1/3): (3 pi / 4)^(2/3) / 2

// Elements of a material's formula unit for the independent-atom Rayleigh form
// factor (n = 0: the analytic F^2 = exp(-q^2/q0^2) and the closed-form total).
struct Elements {
    int n = 0;
    int z[CTD_MAX_ELEMENTS] = {};
    double count[CTD_MAX_ELEMENTS] = {};
};

// message returned by ctd_last_error() on the calling thread (ctd_capi.cu)
void set_error(const char *msg);

// ---- host physics (ctd_physics.cpp) ----
double sigma_kn(double e_kev);
double mu_pe(const ctd_material &m, double e_kev);
double mu_compton(const ctd_material &m, double e_kev);
double mu_rayleigh(const ctd_material &m, double e_kev);
double sigma_wh(double e_kev, double sq0);
double mu_compton_wh(const ctd_material &m, double e_kev);
// independent-atom Rayleigh: total per formula unit (cm^2) and mass attenuation (cm^2/g)
double sigma_rayleigh_iaa(const Elements &el, double e_kev);
double mu_rayleigh_iaa(const ctd_material &m, const Elements &el, double e_kev);

// Node-table columns of one material: out[j*3 + c] the cumulative mass attenuation
// (photoelectric, + Compton, + Rayleigh) at node e_min + j; el.n > 0 gives the
// independent-atom Rayleigh total.
void material_columns(const ctd_material &mat, const Elements &el, int e_min, int n_e, int compton_model,
                      double *out);
// mmax[j]: the majorant scale * max over present materials of rho_max[m] * cum[(m*n_e + j)*3 + 2]
void build_majorant(const std::vector<double> &cum, const std::vector<double> &rho_max, const std::vector<int> &present,
                    int n_e, double scale, std::vector<double> &mmax);
// Inverse-cdf surface rows for node energies e_min..e_min+n_e-1: kind 0 Klein-Nishina,
// 1 Rayleigh of form-factor width q0, 2 Waller-Hartree of scattering-function width q0,
// 3 Rayleigh with the independent-atom form factor of *el.
void build_surface(int kind, double q0, const Elements *el, int e_min, int n_e, int n_zeta, double *out);
// Walker alias table of n intensities (Vose's construction): thr[k] = floor(p 2^32)
// of the kept share of column k, alias[k] the beamlet it borrows from; false if
// the intensities are unusable.
bool alias_build(int n, const double *f, uint32_t *thr, int32_t *alias);
// Largest-remainder allocation; false if the weights are unusable.
bool allocate(uint64_t n, const std::vector<double> &w, std::vector<uint64_t> &out);

// ---- device-side parameter block of one transport launch ----
struct DeviceCounts {
    unsigned long long n[10];   // pe, compton, rayleigh, fictitious, escaped, missed, cutoff, terminated, aborted, steps
    unsigned long long e_fix[4];  // emitted lo, hi, escaped lo, hi: keV * 2^23 as 128-bit integers
};

// keV from a 128-bit fixed-point total (lo, hi) in units of 2^-23 keV
inline double fixed_kev(unsigned long long lo, unsigned long long hi)
{
    return static_cast<double>(hi) * 2199023255552.0 + static_cast<double>(lo) * (1.0 / 8388608.0);
}

enum { kCntPe = 0, kCntCompton, kCntRayleigh, kCntFict, kCntEscaped, kCntMissed, kCntCutoff,
       kCntTerminated, kCntAborted, kCntSteps };

// One request's share of a transport launch.  A single-request launch passes
// it by value (the kernel's parameter space); a multi-request launch passes an
// array of them in device memory, and each warp copies the entry of the
// request it is working on into shared memory.
struct alignas(16) RequestDesc {
    const uint32_t *vox;         // [nvox] material and density of each voxel, one word (kRhoExpBias)
    const void *unused;          // keeps the descriptor a whole number of 16-byte words
    const float *tab;            // [n_mat][n_e][4]: c1, c2, c3 (cm^2/g), c3[j+1] - c3[j] in binary32
    const float *mmax;           // [n_e] majorant mu_max(E), 1/cm
    // R and C surfaces as cells of 4 floats, [n_e - 1][n_zeta - 1] per surface: cell (j, i)
    // holds S[j][i], S[j][i+1], S[j+1][i], S[j+1][i+1], the corners of one bilinear lookup
    const float *rsurf;          // [n_mat] surfaces of cells
    const float *csurf;          // [n_c] surfaces of cells, material m at m * cs_stride cells
    const uint64_t *pref;        // [nbins+1] bin starts inside the batch
    const float *bin_lo;         // [nbins]
    const float *bin_hi;         // [nbins]
    const float *cb;             // [n_proj]
    const float *sb;             // [n_proj]
    const float *zb;             // [n_proj] source height of each projection (helical)
    double *tally;               // [nvox] keV
    DeviceCounts *counts;
    unsigned long long *work;    // claim counter over [local_begin, local_end)
    uint64_t seed;
    uint64_t h_base;             // global index of local index 0 (first history of the batch)
    uint64_t local_begin, local_end;
    int n_mat;
    int nbins;
    int nx, ny, nz;
    float fnx, fny, fnz;         // nx, ny, nz as binary32 (the escape test's bounds)
    float bx0, by0, bz0, bx1, by1, bz1;
    float ix, iy, iz;
    int src_kind, n_proj, continuous;
    float D, D2, ulo, uw, vlo, vw, a0t, awt;
    float hz0, hdz;              // z0 and z1 - z0 of a continuous helical trajectory
    int mode, max_real;
    int cs_stride;               // 0 (one Klein-Nishina surface) or (n_e - 1)(n_zeta - 1) (Waller-Hartree)
    const uint32_t *fl_thr;      // [fl_n] fluence-map alias thresholds (fl_n = 0: no map)
    const int32_t *fl_alias;     // [fl_n]
    int fl_n, fl_nu;
    float fl_du, fl_dv;          // beamlet size at the centre plane, cm
    uint64_t fl_magic;           // floor(2^40 / fl_nu) + 1: I / fl_nu = (I fl_magic) >> 40 for I < 2^24, fl_nu < 2^16
    uint32_t rk[20];             // Philox round keys of seed: (lo, hi) + r (Weyl constants), r = 0..9
};

// blocks copy a descriptor into shared memory in 16-byte words
static_assert(sizeof(RequestDesc) % 16 == 0, "RequestDesc must be a whole number of 16-byte words");

constexpr int kMaxPhantomMaterials = 16;

// A voxel's material and density in one 32-bit word, so that a Woodcock step
// makes one gather: the material index in bits 28-31, the density's binary32
// biased exponent less kRhoExpBias in bits 23-27 and its significand in bits
// 0-22; the word's low 28 bits are 0 for density 0.  Exact for densities 0 and
// [2^-18, 2^13) g/cm^3 (biased exponents 109..139).
constexpr uint32_t kRhoExpBias = 108;
constexpr uint32_t kRhoExpLo = 109, kRhoExpHi = 139;

// What a phantom's voxels hold, found on the device when the phantom is created
// (which also packs each voxel's word): the first voxel whose material index is
// out of range and the first whose density is neither 0 nor in [2^-18, 2^13) g/cm^3
// (~0 if none), which materials occur, and the largest density of each (binary32
// bit patterns, which order like the values for non-negative numbers).
struct PhantomScan {
    unsigned long long first_bad_mat, first_bad_rho;
    unsigned int present_mask;
    unsigned int max_bits[kMaxPhantomMaterials];
};
int launch_scan_phantom(const uint8_t *mat, const float *rho, size_t nvox, int n_mat, uint32_t *vox, double *rinv,
                        PhantomScan *out, void *stream);

// What every request of a launch shares: the node grid and the C surface.
struct SharedTables {
    int n_e, n_zeta, e_min;
    int max_n_mat;               // largest n_mat of the launch's requests (shared-memory size)
};

struct LaunchParams {
    SharedTables sh;
    RequestDesc one;             // the request of a single-request launch
    const RequestDesc *reqs;     // [n_req] (multi-request launches; n_req == 0: single)
    int n_req;
    int chunk;                   // histories a warp claims at a time
    int flight_cap;              // Woodcock flights a lane takes before yielding to the warp
    int any_fluence;             // multi-request launches: some request has a fluence map
    // per-history records of a trace launch (single request; nullptr otherwise):
    // record i is history trace_h0 + i, for i < trace_n
    uint4 *trace;
    uint64_t trace_h0, trace_n;
};

// Per-history record of a trace launch (16 bytes): x = end code + 1 in bits 0-7
// (0: the history never ended) and the last real interaction's type + 1 in bits
// 8-15 (0: none); y = Woodcock steps; z = voxel of the last real interaction;
// w = binary32 bits of the energy the ending event deposited (keV).
enum { kEndPe = 0, kEndCutoff, kEndEscaped, kEndMissed, kEndTerminated, kEndAborted };

// An L2 access-policy window for a launch: [base, base + bytes) persisting for a
// share hit_ratio of its lines, the rest as usual.
struct L2Window {
    void *base;
    size_t bytes;
    float hit_ratio;
};

// launches (ctd_transport.cu / ctd_stats.cu); win may be null
int launch_transport(const LaunchParams &p, int grid, int block, int threads_per_sm, void *stream,
                     const L2Window *win = nullptr);
size_t transport_smem_bytes(const LaunchParams &p, int threads);
int launch_fold(double *tally, const double *rinv, double *sum_d, double *sum_d2, double *edep, size_t nvox,
                double scale, void *stream);
int launch_finalize(const double *sum_d, const double *sum_d2, int nb, double *dose, double *sd, size_t nvox,
                    void *stream);
int launch_rsd(const double *dose, const double *sd, const float *rho, size_t nvox, double *partials,
               int n_parts, double *result, void *stream);
int launch_sample_mu(const float *surf, int n_zeta, int n_e, int e_min, float e, uint64_t seed, uint64_t n,
                     double *out, void *stream);
int launch_eval_math(int fn, const float *x, float *out, size_t n, void *stream);
int launch_sum(const double *x, size_t n, double *partials, int n_parts, double *result, void *stream);

// one fold over several requests' grids in a single launch; tiles of
// kFoldTile voxels, tile_off[r] = first tile of request r
struct FoldDesc {
    double *tally;
    const double *rinv;          // 1 / rho per voxel (0 where rho = 0)
    double *sum_d, *sum_d2, *edep;
    uint64_t nvox;
    double scale;
};
constexpr int kFoldTile = 4096;
int launch_fold_multi(const FoldDesc *descs, const uint64_t *tile_off, int n, uint64_t total_tiles, void *stream);
int launch_probe(int kind, double *dbuf, float *fbuf, uint8_t *mbuf, float *out, uint32_t n_slots, uint32_t rounds,
                 uint32_t salt, int grid, int block, void *stream);

}  // namespace ctd
