// Internal structures shared by the host scheduler and the kernels of
// libahfgpu (not part of the public C ABI).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "ahf.h"

namespace ahf {

// Device-side view of the caller's particle store.
struct ParticlesDev {
  const void *x, *y, *z, *vx, *vy, *vz, *m;
  const void *u_th;    // gas: specific thermal energy per particle, or NULL
  double m0;
  float m0f;
  int coord_type;
  long long n;
};

// Per-halo descriptor prepared on the host.  Haloes are reordered by size
// class and size; `index` is the caller's position (for the result record).
struct HaloDev {
  long long cfix[3];   // centre in 2^-frac units (mixed precision recentring)
  double c[3];         // centre (FP64 recentring)
  double R2;           // gather radius squared
  float R2lo, R2hi;    // float bounds of R^2 that settle membership without FP64
  long long offset;    // first candidate slot
  long long count;     // candidate slots
  long long gbase;     // first position in the class's flat arrays (the multi-CTA
                       // class's work arrays, the on-chip classes' candidate records)
  long long boxfix;    // periodic box in this halo's 2^-frac units (0 = none)
  int frac;            // fractional bits of this halo's fixed-point offsets
  int index;           // caller's halo index
  float cf[3];         // centre as float (when fast)
  int fast;            // float inputs, no box, float-exact centre: x - c in FP32
};                     // is already the correctly rounded offset

// Fill the device descriptor of one halo (shared by every entry point, so a
// halo gets the same frame whichever way it is submitted).
void fill_halo_dev(const ahf_halo &H, int coord_type, double box, int index, HaloDev &d);

struct FrameDev {
  double box;          // periodic box (0 = none)
};

struct ParamsDev {
  double G, H, delta_rho, r_soft, band;
  float Gf, Hf, r_soft_f, band_f;
  float crit_f;        // delta_rho * 4 pi / 3 as float
  double crit;         // delta_rho * 4 pi / 3
  double inv_crit;     // 1 / crit
  int max_iter;
  int precision;
  int vbulk_initial;   // AHF_VAR_VBULK_INITIAL: v_bulk of the initial set throughout
  int rise_edge;       // AHF_VAR_RISE_EDGE: extent at the rise of the density profile
};

struct OutputsDev {
  ahf_result *res;
  long long *bound_idx;
  void *phi;
  int *removed_iter;
  const long long *member_idx;
  long long n_slots;
  int *err;            // device error word (bit flags, see ERR_*)
};

// Device error bits reported back through the error word.
constexpr int ERR_BAD_INDEX = 1;     // a member index was out of range
constexpr int ERR_TIMEOUT = 2;       // a bounded wait on a tensor copy gave up
constexpr int ERR_CAPACITY = 4;      // a halo exceeded its class capacity

// An exact fixed-point sum of the multi-CTA class: a long long (mixed
// precision) or an __int128 (all-FP64 mode) held in the first bytes.
struct alignas(16) AccSlot {
  long long w[2];
};

// Per-halo state of the multi-CTA class, kept in the context's workspace.
struct GridHaloState {
  unsigned long long mass_max_bits;  // bits of the largest member mass
  unsigned long long mr_max_bits;    // bits of the largest m/r
  unsigned long long mv_max_bits;    // bits of the largest |m v_k|
  long long n_member;
  long long n_alive;                 // members alive at the start of the next pass
  long long part_iter;
  long long band;                    // band tests so far
  long long k_first;                 // first virial crossing (compacted index)
  AccSlot m_tot;                     // exact sum of the alive masses
  AccSlot t_tot;                     // exact sum of m/r over the alive set
  AccSlot mv[3];                     // exact sum of m v over the alive set
  int n_iter;
  int status;
  int active;
  int s_m, s_mr, s_mv;               // fixed-point scales
  int pad0, pad;
  AccSlot rem_mv[3];                 // exact sum m v of what the current pass removed
  long long band_pass;               // band tests of the current pass
  float vbulk[3];                    // v_bulk of the current set (mixed precision)
  float pad2;
  double vbulk_d[3];                 // v_bulk of the current set (all-FP64 mode)
  AccSlot m_init;                    // exact sum of the members' masses (before any pass)
  double mrem;                       // mass the halo lost before the current pass
  double pad3;
};

// What the last pass that tested a sub-tile of the multi-CTA class saw, so
// that a later pass can leave the sub-tile out while none of its members can
// be removed or fall in the band (a bound on how far phi and |u| can have
// moved since; the pass then re-tests nothing that could change).
struct SkipRec {
  float margin;  // min over the members it left alive of 2|phi| (1 - band - 2^-16) - |u|^2 (+ 2 u_th),
                 // rounded down; +inf when none is left
  float umax;    // max |u| over them, rounded up
  float rin;     // |r| of the sub-tile's first element, rounded down (no member is closer)
  float vb[3];   // v_bulk of that pass
  double mrem;   // mass the halo had lost before that pass
};

// Device control words of one multi-CTA call.
struct GridCtl {
  int work_n[2];                     // sub-tiles to process in the passes of each parity
  int pad0[2];
  unsigned long long key_or, key_and;  // OR and AND of every radius key
  int pad[8];
};

// Record a static message as the thread's last error (no allocation).
void set_last_error_static(const char *msg);
// Record a formatted message as the thread's last error and return `code`.
int set_last_error_fmt(int code, const char *fmt, ...);

// ---- launchers (defined in the .cu files) -----------------------------------

// Profile rows requested from the unbinding kernels themselves.
// Per-bin tables of a profile call (3 n doubles, from profile_bin_tables):
//   [0, n)   f_b = f^(1 - b/n), the edge e_b = r_out f_b (e_n = r_out)
//   [n, 2n)  1 / (4 pi / 3 (f_{b+1}^3 - f_b^3)): shell volume = r_out^3 / this
//   [2n, 3n) 1 / f_{b+1}
void profile_bin_tables(int n_bins, double r_min_frac, double *t);

struct ProfileRows {
  double *prof;              // [n_halos][n_bins][4] (caller order), NULL = none
  const double *factor;      // the bin tables (3 n_bins doubles)
  const float *factor_f;     // the same rounded to float
  int n_bins;
};

struct OnchipLaunch {
  ParticlesDev p;
  FrameDev frame;
  ParamsDev prm;
  OutputsDev out;
  const HaloDev *halos;  // this class's haloes, largest first
  int n_halos;
  int *queue;            // work counter (zeroed by the launcher)
  ProfileRows rows;      // rows.prof == NULL: no profile from this launch
  long long *trace;      // [halo index][AHF_TRACE_FIELDS] or NULL
  int variant;           // phase index of this class (for the trace)
  // candidate records, two per candidate from 2 * halos[k].gbase on:
  // (d_x, d_y, d_z, m) and (v_x, v_y, v_z, 0) as the gather computed them,
  // read back in radial order by the fill and the removals (two 16-byte
  // loads in place of seven scattered 4-byte ones).  NULL: both read the
  // particle store again.
  float4 *rec;
};

// Warp class: one warp per halo of at most warp_capacity() candidates.
int warp_capacity();
int warp_max_grid(int device);
int warp_halos_per_cta();
cudaError_t launch_warp(const OnchipLaunch &L, int grid, cudaStream_t s);

// Shared-memory CTA / cluster variants 0..5: candidate capacity, CTAs per cluster.
int onchip_capacity(int variant);
int onchip_cluster_size(int variant);
// Launch the on-chip class (variant chosen by the scheduler).
cudaError_t launch_onchip(const OnchipLaunch &L, int variant, int grid, cudaStream_t s);
int onchip_max_grid(int variant, int device);

struct GridLaunch {
  // the radial-order stream (w, r) as a 2-D tensor of 8-element rows (128
  // bytes), for the passes' tensor copies into shared memory (mixed mode)
  alignas(64) CUtensorMap wr_map;
  int use_tma;             // the passes stage sub-tiles through wr_map
  int tma_grid;            // CTAs of that pass kernel
  long long wait_limit;    // polls of a copy's barrier before giving up (ERR_TIMEOUT)
  ParticlesDev p;
  FrameDev frame;
  ParamsDev prm;
  OutputsDev out;
  HaloDev* halos;          // device copy of the class's haloes
  int n_halos;
  long long n_flat;        // sum of candidate counts of the class
  GridHaloState* state;    // n_halos
  int fp64;                // 0: mixed precision (float), 1: all-FP64 (double)
  GridCtl* ctl;
  // flat arrays (n_flat each unless noted); element types follow fp64
  void* rec;               // 2 per candidate: (w.x, w.y, w.z, r), (v.x, v.y, v.z, m)
                           // as float4 / 4 doubles, by candidate position
  void *key_a, *key_b;     // radius keys: uint32 / uint64
  uint32_t *val_a, *val_b; // candidate positions riding along the sort
  void* wr;                // radial order: (w.x, w.y, w.z, r), r's sign bit = removed
  void* ms;                // radial order masses (float / double), NULL for a uniform mass
  void* uth;               // gas: thermal energy in radial order (float / double), or NULL
  uint32_t* val_x;         // radial order -> candidate position
  void* mc;                // compacted inclusive mass (final pass): long long / __int128
  void* rc;                // compacted radius (final pass): float / double
  // tiles
  int n_tiles;
  int2* tile_range;        // (first flat index, length)
  int* tile_halo;
  int* halo_tile0;         // first tile of each halo (n_halos + 1)
  uint32_t* tile_hist;     // n_tiles * 256, per halo digit-major
  uint32_t* digit_base;    // n_halos * 256
  int* big_halos;          // haloes of more than 256 tiles (digit scans spread over CTAs)
  int n_big;
  int max_halo_tiles;      // tiles of the largest halo
  // per sub-tile of GRID_SUB elements (GRID_TILE / GRID_SUB per tile), two
  // copies by pass parity (pass p reads copy p & 1 and writes the other): the
  // exact sums (m, m/r as long long / __int128) and count of its alive members
  void *agg_m, *agg_r;
  int* agg_c;
  // per tile: exclusive prefix of the alive sums over the halo's tiles before
  // it (for the next pass, then the final one)
  void *pre_m, *pre_r;
  long long* pre_c;
  AccSlot* tile_mv;        // [n_tiles][3]: sum m v of each tile's members (initial set)
  SkipRec* skip;           // [n_tiles * GRID_TILE / GRID_SUB]: the last test of each sub-tile
  uint8_t* rem_mask;       // [n_tiles * GRID_TILE / GRID_SUB][32]: removal flags of the last
                           // pass, one byte per lane (bit i: the lane's element i)
  int4* work;              // [2][n_tiles * GRID_TILE / GRID_SUB]: the sub-tiles of the active
                           // haloes for the passes of each parity: (sub-tile, halo, first
                           // flat element, members in it)
  int iter_grid;           // CTAs of the persistent iteration pass
  int sort_passes;         // radix passes the last grid_sort launched
  int sort_launches;       // and its kernel launches
  ProfileRows rows;        // rows.prof != NULL: profile rows from the final pass
};

constexpr int GRID_TILE = 2048;
constexpr int GRID_THREADS = 256;
constexpr int GRID_SUB = 256;      // elements of a sub-tile (one warp's share of a pass)

// CTAs of the multi-CTA class's persistent iteration pass that fit on
// `device` at once.
int grid_iter_grid(int device, int fp64);
int grid_tma_grid(int device);
// Fill L.wr_map for the stream L.wr of n_rows 8-element rows; false if the
// tensor map cannot be made (the passes then read the stream directly).
bool grid_wr_map(GridLaunch &L, long long n_rows);
cudaError_t grid_prepare(const GridLaunch &L, cudaStream_t s);
// Radix passes over the bits where the keys differ (or_bits ^ and_bits);
// the last pass also lays out the radial-order streams.  Then the sums of
// the initial set.
cudaError_t grid_sort(GridLaunch &L, cudaStream_t s, unsigned long long or_bits, unsigned long long and_bits);
// One unbinding pass over every active halo (pass = iteration number).
cudaError_t grid_iterate(const GridLaunch &L, int pass, cudaStream_t s);
// Bound lists, phi, virial crossing, records and (rows.prof) profile rows.
cudaError_t grid_finish(const GridLaunch &L, cudaStream_t s);

struct ProfileLaunch {
  ParticlesDev p;
  FrameDev frame;
  ParamsDev prm;
  OutputsDev out;
  const HaloDev *halos;    // all haloes (caller order)
  int n_halos;
  const ahf_result *res;
  const long long *bound_idx;
  int n_bins;
  double r_min_frac;
  double *prof;
  long long *chunk_acc;    // workspace: per chunk (inner mass, inner count, per bin count and mass)
  int *chunk_halo;         // chunk -> halo
  long long *chunk_start;  // chunk -> first position in the halo's bound list
  const double *edge_factor;  // the bin tables (3 n_bins doubles)
  const float *edge_factor_f; // the same rounded to float
  int n_chunks;
  int n_multi;             // haloes held by more than one chunk
};
constexpr int PROFILE_CHUNK = 4096;
int profile_max_bins();
cudaError_t launch_profile(const ProfileLaunch &L, const int *halo_chunk0, cudaStream_t s);

// Integral properties of bound sets (spin parameter, energies, rotation-curve
// peak), chunked like the profile: per chunk partial moments, a second pass
// for the inclusive-mass prefix, then one combine per halo.
constexpr int PROPS_CHUNK = 4096;
constexpr int PROPS_PART = 20;           // doubles of per-chunk partials
struct PropsLaunch {
  ParticlesDev p;
  FrameDev frame;
  double G, H;
  const HaloDev *halos;                  // caller order
  int n_halos;
  const ahf_result *res;
  const long long *bound_idx;            // particle indices, radial order per halo
  const void *phi;                       // float (mixed) or double (FP64) per slot
  int phi_f64;
  const int *chunk_halo;
  const long long *chunk_start;
  const int *halo_chunk0;                // [n_halos + 1]
  int n_chunks;
  double *part;                          // [n_chunks][PROPS_PART]
  double *props;                         // [n_halos][AHF_PROP_FIELDS]
};
cudaError_t launch_properties(const PropsLaunch &L, cudaStream_t s);

// Hosts and subhaloes in dependency order: the kernels around each level.
struct HierLaunch {
  const ahf_halo *halos;           // device copy of the caller's descriptors
  const int *level;                // caller indices of this level's haloes
  const long long *member_idx;     // caller's member list or NULL
  long long n_particles;
  long long *owner;                // [n_particles]: level rank << 32 | halo, -1 none
  const int *anc;                  // [n_halos]: ancestor on this level, -1
  long long *members;              // [n_slots] compacted member lists
  long long *cand_map;             // [n_slots] compacted position -> candidate slot
  long long *kept;                 // [n_level] kept candidates
  const ahf_result *res_level;     // [n_level]
  ahf_result *res;                 // caller's records
  const int *rem_level;            // [n_slots] removal iterations by compacted slot
  int *removed_iter;               // caller's, or NULL
  const long long *bound_idx;      // caller's
  int rank;                        // 0 for the deepest level, growing outwards
};
cudaError_t launch_hier_compact(const HierLaunch &L, int n_level, cudaStream_t s);
cudaError_t launch_hier_scatter(const HierLaunch &L, int n_level, cudaStream_t s);

// Cross-identification of two catalogues by xi = N_shared^2 / (N_1 N_2).
constexpr int MATCH_TABLE = 2048;        // distinct second-catalogue haloes one halo may meet
constexpr int ERR_ID_RANGE = 8;          // a particle id outside [0, n_ids)
constexpr int ERR_SHARED_ID = 16;        // a particle in two haloes of the second catalogue
constexpr int ERR_MATCH_TABLE = 32;      // a halo met more than MATCH_TABLE haloes
struct MatchLaunch {
  long long n_ids;
  const long long *ids_a, *off_a, *cnt_a;
  int n_a;
  const long long *ids_b, *off_b, *cnt_b;
  int n_b;
  int *label;                            // [n_ids] workspace
  int *err;
  long long *best, *shared;
  double *xi;
};
cudaError_t launch_match(const MatchLaunch &L, cudaStream_t s);

}  // namespace ahf
