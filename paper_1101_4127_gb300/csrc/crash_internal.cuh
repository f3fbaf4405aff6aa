// crash_internal.cuh -- device data layout and kernel interfaces shared by
// the CUDA translation units of libcrash (not part of the public ABI).
//
// HBM layout (all boxes of a batch concatenated, x fastest inside a box):
//   nH      float  [cells]          hydrogen density (static input)
//   x_HII, x_HeII, x_HeIII, T  double [cells]  state (SoA, coalesced per-cell kernels)
//   abs64   double4-like [cells]    n_HI, n_HeI, n_HeII, 0 frozen per step (FP64 form)
//   abs32   float4  [cells]         the same in FP32 (mixed form)
//   dep     int64 x4 [cells]        dep_HI, dep_HeI, dep_HeII, dep_E (one 32-byte sector per cell)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "crash.h"

#define CRASH_MAX_BINS 16
#define CRASH_MAX_BOXES 4096

// Per-box constants (uploaded when sources or per-step plans change).
struct BoxMeta {
  int nx, ny, nz;
  int isothermal;
  int64_t cell_off;    // first cell of the box in the concatenated arrays
  int64_t ncell;
  double dl;           // cell edge, cm
  float dlf;           // the same in FP32 (mixed form)
  double he;           // n_He / n_H
  double T_cmb;        // 0 => Compton off
  uint64_t seed;
  int caseB;
  int src_off;         // sources [src_off, src_off + n_src)
  int n_src;
  int heatF;           // heat unit 2^heatF eV (per photon quantum)
  double ndot_sum;     // photon rate of all the box's sources, summed in source order
  // per-step packet plan
  uint64_t pkts_per_src;   // N_s = packets_per_step / n_src
  uint32_t win_lo, win_hi; // traced packet ids [win_lo, win_hi) per source
  int64_t pkt_off;         // first global packet slot of this box in the launch
  int64_t pkt_count;       // n_src * (win_hi - win_lo)
  // wavefront re-sort: keys of this box start at bucket_off; a key is
  // morton(ix >> 3, iy >> 3, iz >> 3) (bucket_bits bits per axis) * 8 + octant
  int64_t bucket_off;
  int bucket_bits;
  // tile passes: keys of this box start at tile_off; a key is
  // morton(ix >> 4, iy >> 4, iz >> 4) (tile_bits bits per axis) * 8 + octant
  int64_t tile_off;
  int tile_bits;
  int max_iter;            // bound on the DDA steps of one packet: nx + ny + nz + 3, or
                           // 2 L + 4 in a periodic box whose packets travel L cells
  double f_rec;            // > 0: diffuse recombination field with this re-emission threshold
  int coupling;            // 1: photon-conserving transport -> chemistry coupling
  int periodic;            // 1: periodic box, walks end after c dt
  float path_cells32;      // periodic: c dt / dl of this step in FP32 (mixed form)
  double uv[3];            // uniform background photo-ionisations per atom (s^-1): H I, He I, He II
  double uve[3];           // heat per such photo-ionisation (eV)
};

// speed of light (cm/s): the periodic box's light-travel distance per step
#define CRASH_C_LIGHT 2.99792458e10

// Cross sections and heating weights per species and bin (passed by value;
// kernel parameters live in the constant bank).
struct BinTables {
  int n_bins;
  double sigma[3][CRASH_MAX_BINS];   // cm^2
  double wheat[3][CRASH_MAX_BINS];   // (E_j - E_th,s) / 2^F, or 0 below threshold
  float sigma32[3][CRASH_MAX_BINS];
  float wheat32[3][CRASH_MAX_BINS];
  float sigma32_max[3];              // largest sigma32 of each species over the bins
  float sw32[3][CRASH_MAX_BINS];     // sigma32 * wheat32 (FP32 product): heating weight per unit t_s
};

struct StepArgs {
  const BoxMeta* boxes;
  int n_boxes;
  unsigned long long* step_dev;   // step index (Philox counter word), advanced on the device
  double dt;
  int64_t total_packets;
  // sources
  const double* src_pos;     // [n_src_total][3]
  const float* src_pos32;    // [n_src_total][3] the same in FP32 (mixed form)
  const int* src_cell;       // [n_src_total][3] cell of each source
  const double* src_ndot;    // [n_src_total]
  const double* src_frac;    // [n_src_total][n_bins]
  int64_t* src_base;         // [n_src_total][n_bins]  per-packet content base (written per step)
  int64_t* src_rem;          // [n_src_total][n_bins]  packets p < rem get one more quantum
  int* box_E;                // [n_boxes] photon quantum exponent this step
  int n_src_total;
  // grid
  const float* nH;
  double* xHII; double* xHeII; double* xHeIII; double* T;
  double* abs64;             // [cells][4]
  float* abs32;              // [cells][4]
  unsigned long long* dep;   // [cells][4]
  int64_t n_cells_total;
  // budget [n_boxes][8] and device error word
  unsigned long long* budget;
  unsigned long long* work;  // work counter of the persistent chemistry kernel
  int64_t n_tile_keys;       // tile-pass sort keys over all boxes
  int max_tiles;             // bound on the tiles one packet crosses
  int* err;
  // options
  int any_he;                // some box has helium (selects the H+He kernels)
  int any_heat;              // some box evolves T (selects the heating deposit)
  int any_periodic;          // some box is periodic (selects the wrapping walks)
  int max_iter_step;         // largest per-box DDA bound of this step
  int chemistry;
  int fp32_rates;            // mixed form: rate fits evaluated in FP32
  double chem_eps;
  int chem_max_sub;
  int cool_mask;
  // diffuse recombination field (some box has f_rec > 0)
  int any_rec;
  double* rec;               // [3][cells] ground-state recombination photons (H I, He I, He II)
  long long* rec_list;       // [cells][4] re-emitting cell, then quanta of H I, He I, He II photons
  unsigned* rec_count;       // entries of rec_list this step
  unsigned long long* rec_rmax;  // [n_boxes] bits of the largest count over threshold (>= 0 doubles)
  int rec_bin[3];            // bin of each species' re-emitted photons, -1 => none
};

// device error bits
enum { ERR_DDA_LIMIT = 1, ERR_DIRECTION = 2, ERR_QUEUE = 4, ERR_WATCHDOG = 8 };

// launchers implemented in the kernel translation units
void launch_prep(const StepArgs& a, int precision, cudaStream_t s);
void launch_budget(const StepArgs& a, const BinTables& t, cudaStream_t s);
void launch_trace_fp64(const StepArgs& a, const BinTables& t, int block, cudaStream_t s);
void launch_chemistry(const StepArgs& a, cudaStream_t s);
// diffuse recombination field: pick this step's re-emitting cells (and
// restart their counts), then trace one packet per cell in either form
void launch_rec_max(const StepArgs& a, cudaStream_t s);   // before launch_budget
void launch_rec_select(const StepArgs& a, cudaStream_t s);
void launch_rec_fp64(const StepArgs& a, const BinTables& t, cudaStream_t s);
int launch_rec_mixed(const StepArgs& a, const BinTables& t, cudaStream_t s);

// Mixed-form transport.  Returns the number of kernels launched (>= 0) or
// -1 on a launch error.  ev/ev_used: optional event pairs recorded around
// the transport kernels.  max_iter: largest per-box DDA bound.
typedef std::vector<std::pair<cudaEvent_t, cudaEvent_t>> EventPairs;
int launch_trace_mixed(const StepArgs& a, const BinTables& t, const crash_run_opts& o,
                       void* wf_state, int max_iter, cudaStream_t s, EventPairs* ev, int* ev_used);

// Mixed-form wavefront over caller-provided record buffers (no allocation,
// no re-sort): rec0/rec1 hold cap records each, count holds 4 counters.
int launch_trace_mixed_external(const StepArgs& a, const BinTables& t, const crash_run_opts& o,
                                char* rec0, char* rec1, unsigned* count, int64_t cap, int max_iter,
                                cudaStream_t s);
// cross sections, heating weights and heat exponent of a bin table (host)
void cross_sections(int nb, const double* E, BinTables& t, int& heatF);

// wavefront workspace (mixed form): capacity in packets, number of sort keys
void* wavefront_create(int64_t capacity, int64_t n_keys, int n_bins, cudaError_t* err);
void wavefront_destroy(void* w);
int64_t wavefront_capacity(void* w);
