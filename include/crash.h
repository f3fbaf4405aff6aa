/*
 * crash.h -- C ABI of the GB300 (sm_103a) Monte-Carlo radiative-transfer step.
 *
 * The library runs the data-parallel hot path of a CRASH2-style step
 * (arXiv:1101.4127, Sec. 2 and Sec. 3.2) on one GPU:
 *   emission of photon packets from point sources (Sec. 2: coloured packets,
 *   N_p/N_t packets per source per step, Sec. 3.2), cell-by-cell propagation
 *   through a 3D Cartesian grid with attenuation by the H I / He I / He II
 *   optical depth (Sec. 2, Eq. 1) and deposition of the absorbed photons in
 *   the crossed cells, followed by the per-cell ionisation network and
 *   temperature update (Sec. 2; sub-sampled as in Sec. 3.2).
 *
 * Conventions shared by every call:
 *   - Grids are nx*ny*nz cubic cells stored x fastest: cell (i,j,k) has the
 *     linear index i + nx*(j + ny*k).  Positions are in grid units: cell
 *     (i,j,k) spans [i,i+1) x [j,j+1) x [k,k+1).
 *   - Units are cgs: cm, s, cm^-3, K, photons/s, eV for photon energies.
 *   - Every pointer argument is a HOST pointer unless the name ends in _dev.
 *     The caller owns its buffers; the library copies what it needs before
 *     the call returns.  The context owns all device memory and one CUDA
 *     stream; nothing is shared between contexts.
 *   - Functions never abort.  They return a crash_status and, on failure,
 *     leave a message for crash_last_error().  A CRASH_ERR_CUDA or
 *     CRASH_ERR_TIMEOUT result leaves the context usable only for
 *     crash_read_fields and crash_free.
 *   - The transported photons are integers in units of a per-step quantum
 *     q = 2^E (E chosen per box and step so that the step's photons of all
 *     the box's sources, sum(ndot) * dt / q, are at most 2^62), so emitted =
 *     absorbed + escaped holds exactly.
 */
#ifndef CRASH_H
#define CRASH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crash_ctx crash_ctx;   /* opaque; owns all device memory */

typedef enum {
  CRASH_OK = 0,
  CRASH_ERR_ARG = -1,        /* invalid argument (message says which) */
  CRASH_ERR_OOM = -2,        /* device or host allocation failed */
  CRASH_ERR_CUDA = -3,       /* a CUDA call or kernel failed */
  CRASH_ERR_OVERFLOW = -4,   /* a capacity (packets, bins, queue) would be exceeded */
  CRASH_ERR_TIMEOUT = -5,    /* a device-side bounded loop hit its limit */
  CRASH_ERR_STATE = -6       /* call out of order (e.g. crash_step before sources) */
} crash_status;

typedef enum {
  CRASH_FP64_PLAIN = 0,      /* FP64 transport, bit-exact with the FP64 specification */
  CRASH_MIXED = 1            /* FP32 traversal/attenuation, int64 deposits, FP64 chemistry */
} crash_precision;

/* Field ids for crash_read_fields / crash_write_fields. */
typedef enum {
  CRASH_F_XHII = 0, CRASH_F_XHEII = 1, CRASH_F_XHEIII = 2, CRASH_F_T = 3, /* double per cell (r/w) */
  CRASH_F_DEP_HI = 4, CRASH_F_DEP_HEI = 5, CRASH_F_DEP_HEII = 6,          /* int64 per cell, last step */
  CRASH_F_DEP_E = 7,        /* int64 per cell: excess energy in units of q * 2^F eV */
  CRASH_F_BUDGET = 8,       /* int64[8]: emitted, absorbed, escaped, crossings,
                               packets traced, quantum exponent E, heat exponent F,
                               chemistry sub-steps (all for the last step) */
  CRASH_F_NH = 9,           /* double per cell: n_H (read only) */
  CRASH_F_TOTALS = 10,      /* int64[8]: slots 0-4 and 7 of CRASH_F_BUDGET summed over all
                               steps since the context was created (slots 5, 6: last step) */
  /* double per cell (r/w), only when the diffuse field is on (f_rec > 0):
     photons of recombinations to the ground state of H I, He I and He II
     counted since the cell last re-emitted them */
  CRASH_F_REC_HI = 11, CRASH_F_REC_HEI = 12, CRASH_F_REC_HEII = 13
} crash_field;

/* One grid and its initial state.  Section 2 of the paper: a static H/He
   density field on a Cartesian grid whose ionisation fractions and
   temperature evolve. */
typedef struct {
  int nx, ny, nz;            /* cells per axis, each >= 1 */
  double box_cm;             /* length of the x edge; cell edge dl = box_cm / nx */
  const float* n_H;          /* nx*ny*nz hydrogen densities (cm^-3); NULL => n_H0 everywhere */
  double n_H0;
  double he_over_h;          /* helium-to-hydrogen number ratio; 0 => pure hydrogen */
  const double *x_HII, *x_HeII, *x_HeIII, *T;   /* initial state per cell; NULL => uniform value */
  double x_HII0, x_HeII0, x_HeIII0, T0;
  int isothermal;            /* 1: T stays fixed (no heating deposit, no T update) */
  int caseB;                 /* 1: case-B recombination (on-the-spot), 0: case A */
  double z_compton;          /* redshift of the CMB for Compton exchange; < 0 => off */
  uint64_t seed;             /* Philox key of this grid */
  int precision;             /* crash_precision; must be equal for all boxes of a batch */
  double f_rec;              /* diffuse recombination radiation (Sec. 2): 0 => off (on-the-spot
                                recombination as caseB says).  > 0 => case A recombination;
                                recombinations to the ground state are counted per cell and
                                species, and at the start of a step every cell where a
                                species' count reached f_rec times that element's atoms in
                                the cell re-emits it as one isotropic packet from a uniform
                                point of the cell, in the lowest bin at or above the
                                species' threshold; the count then restarts.  The photon
                                quantum of the step also keeps (cells of the box) x (largest
                                count over its threshold) below 2^62 quanta, and then takes
                                one more bit, so sources plus re-emission fit in int64. */
  int coupling;              /* transport -> chemistry (Sec. 2 couples the absorbed photons to
                                the network; the form is a reading):
                                0 = photo-ionisation rate per absorber frozen at the start of
                                the step, Gamma_s = dep_s q / (dt n_s V) (default);
                                1 = photon-conserving: the step's absorbed photons ionise at a
                                constant rate, dep_s q / (dt V) atoms per cm^3 and s, in
                                each chemistry sub-step at most the atoms of the species
                                present (the photons beyond are lost); photo-heating at the
                                deposited rate. */
  int periodic;              /* 1: periodic box (Sec. 2): a packet crossing a face re-enters
                                through the opposite one; its walk ends after the distance
                                light travels in the step, c dt (at most 2^29 cells), and
                                what it still holds then is counted as escaped.  Periodic
                                boxes trace every packet to its end in its own thread (the
                                mixed form's wavefront keeps no path budget). */
  double uv_rate[3];         /* uniform background (Sec. 2 "background field"; the paper
                                gives neither its intensity nor its spectrum, so it is
                                taken as given rates): photo-ionisations per atom of H I,
                                He I and He II and second, the same in every cell, not
                                attenuated, added to the rates from the deposits in the
                                per-cell update (>= 0, finite; 0 = off, the default) */
  double uv_heat_eV[3];      /* heat each such photo-ionisation leaves in the gas, eV (>= 0) */
} crash_grid_desc;

/* Run options (crash_default_opts fills the defaults). */
typedef struct {
  int chemistry;             /* 1: per-cell update after transport (default); 0: transport only */
  uint32_t pkt_begin, pkt_end; /* trace only packet ids p in [pkt_begin, pkt_end) of each source
                                  (default 0, 0xFFFFFFFF: all); contents are those of the full step */
  double chem_eps;           /* allowed relative change per chemistry sub-step (default 0.1) */
  int chem_max_sub;          /* sub-step cap per cell and step (default 10000) */
  int cool_mask;             /* processes on: 1 coll. excitation, 2 coll. ionisation, 4 recombination,
                                8 bremsstrahlung, 16 Compton, 32 dielectronic (default 63) */
  int block_size;            /* threads per block of the transport kernels (0 = tuned/default) */
  int seg_per_iter;          /* mixed form: crossings per packet per wavefront pass (0 = tuned) */
  int resort_interval;       /* mixed form: wavefront passes between Morton re-sorts (0 = tuned,
                                <0 = never) */
  int wavefront;             /* mixed form: 1 = packet-queue wavefront, 0 = one thread per packet */
  int use_graph;             /* 1: capture each step in a CUDA graph and replay it */
  int timing;                /* 1: record CUDA events around the transport launches */
  int reg_cap;               /* mixed form: 1 = transport kernels capped at 64 registers
                                (more resident warps), 0 = uncapped (tuned/default) */
  int tile;                  /* mixed form: 1 = tile passes (packets sorted into 16^3-cell
                                tiles; a tile's absorbers and deposits held in shared memory
                                while its packets cross it); 0 = passes of seg_per_iter cells
                                over global memory */
  int pass_limit;            /* mixed form: at most this many wavefront passes per chunk
                                (0 = as many as the grid needs).  A packet still alive after
                                the last pass is a device-side limit: the next synchronising
                                call returns CRASH_ERR_TIMEOUT. */
  int sort_curve;            /* mixed form: order of the buckets in the re-sort key,
                                0 = Morton (Z) curve, 1 = Hilbert curve; tile passes
                                (tile = 1) always key by Morton tiles.  Results do not
                                depend on it (only the order packets are traced in). */
  int chunk_packets;         /* mixed form: packets per wavefront chunk (0 = 2^28); a step
                                with more packets runs chunk after chunk through one queue.
                                Results do not depend on it. */
  int persistent;            /* mixed form, wavefront without tiles: 1 = the whole transport
                                of a step in one cooperative launch whose blocks stay
                                resident and meet at grid barriers between passes and
                                re-sort phases (default); 0 = one launch per pass and per
                                re-sort phase.  Every barrier wait is bounded (30 s), after
                                which the step reports CRASH_ERR_TIMEOUT.  Results do not
                                depend on it. */
} crash_run_opts;

void crash_default_opts(crash_run_opts* o);

/* Device memory of a context may be capped with the environment variable
   CRASH_DEVICE_MEMORY_CAP (bytes): creation, sources or a step whose
   allocations would exceed it fail with CRASH_ERR_OOM and allocate nothing. */

/* Create a context holding one grid (equivalent to a batch of one). */
crash_status crash_init_grid(const crash_grid_desc* desc, crash_ctx** out);

/* Create a context holding n_boxes independent grids that step together
   (the batched form).  Each box keeps its own seed, sources and budget. */
crash_status crash_init_batch(int n_boxes, const crash_grid_desc* descs, crash_ctx** out);

/* Sources of box `box` (Sec. 2: point sources with luminosity and spectrum).
   pos_cells: n_src*3 grid-unit positions inside [0,nx)x[0,ny)x[0,nz);
   ndot: n_src photon rates (photons/s, >= 0);
   bin_eV: n_bins bin energies (eV, > 0), 1 <= n_bins <= 16, identical for all boxes;
   bin_frac: n_src*n_bins photon-number fractions per source (>= 0; the last bin
   takes what the cumulative fractions leave).  Replaces earlier sources. */
crash_status crash_add_sources(crash_ctx* ctx, int n_src, const double* pos_cells,
                               const double* ndot, int n_bins, const double* bin_eV,
                               const double* bin_frac);
crash_status crash_add_sources_box(crash_ctx* ctx, int box, int n_src, const double* pos_cells,
                                   const double* ndot, int n_bins, const double* bin_eV,
                                   const double* bin_frac);

crash_status crash_set_options(crash_ctx* ctx, const crash_run_opts* opts);
/* Copy the context's current options (after crash_autotune: the chosen ones)
   to *opts. */
crash_status crash_get_options(crash_ctx* ctx, crash_run_opts* opts);

/* One time step of length dt_s (Sec. 2 and Sec. 3.2): every box emits
   packets_per_step packets split equally over its sources (must be a
   multiple of each box's source count), traces them against the absorbers
   frozen at the start of the step, then (if enabled) updates every cell.
   The call is asynchronous on the context stream except for argument checks;
   read_fields and sync wait for it. */
crash_status crash_step(crash_ctx* ctx, double dt_s, uint64_t packets_per_step);
/* Batched form: per-box packet counts (n_boxes entries). */
crash_status crash_step_batch(crash_ctx* ctx, double dt_s, const uint64_t* packets_per_box);

/* Copy a field of box 0 / of box `box` to host memory (size: cells of the box
   times 8 bytes, or 64 bytes for CRASH_F_BUDGET).  Synchronises the stream. */
crash_status crash_read_fields(crash_ctx* ctx, int field_id, void* host_out);
crash_status crash_read_fields_box(crash_ctx* ctx, int box, int field_id, void* host_out);
/* Overwrite a state field (x_HII, x_HeII, x_HeIII or T) of box 0 / `box` from host memory. */
crash_status crash_write_fields(crash_ctx* ctx, int field_id, const void* host_in);
crash_status crash_write_fields_box(crash_ctx* ctx, int box, int field_id, const void* host_in);

/* Device-side checkpoint of the state fields (x_HII, x_HeII, x_HeIII, T)
   and the step index, kept in a snapshot buffer owned by the context
   (allocated by the first save).  op = CRASH_CKPT_SAVE stores the current
   state; CRASH_CKPT_RESTORE_STATE copies the stored fields back and keeps
   the step index running (the next step draws new directions);
   CRASH_CKPT_RESTORE also restores the step index (the next step repeats
   bit for bit).  Asynchronous on the context stream.  Restoring before any
   save is CRASH_ERR_STATE. */
enum { CRASH_CKPT_SAVE = 0, CRASH_CKPT_RESTORE_STATE = 1, CRASH_CKPT_RESTORE = 2 };
crash_status crash_checkpoint(crash_ctx* ctx, int op);

/* Step counter used as the Philox counter word (resume: restore the fields,
   then set the index of the next step). */
crash_status crash_set_step_index(crash_ctx* ctx, uint64_t step);
crash_status crash_sync(crash_ctx* ctx);

/* Event-timed transport: total milliseconds and launch count of the dominant
   transport kernel since the last reset (needs opts.timing = 1). */
crash_status crash_kernel_time(crash_ctx* ctx, double* ms_total, int64_t* launches);
crash_status crash_reset_kernel_time(crash_ctx* ctx);

/* The context's CUDA stream (a cudaStream_t) for callers that time or order
   work around crash_step. */
void* crash_stream(crash_ctx* ctx);

/* Number of kernel launches the context has enqueued since it was created
   (graph replays count the kernels inside the graph). */
int64_t crash_launch_count(crash_ctx* ctx);

/* Autotuner: times transport-only trial steps over block size, crossings
   per pass, re-sort interval, register cap and tile passes (mixed form) on
   the current state, over a window of about 2^26 packet ids, one launch
   per pass; then the fastest once more with Hilbert-ordered re-sort keys,
   and the fastest of those once more as one persistent launch per step
   (opts.persistent); the state, the diffuse field's counts and the step
   index are restored afterwards.  Stores the fastest in the context's
   options (persistent included) and returns the chosen values (outputs may
   be NULL). */
crash_status crash_autotune(crash_ctx* ctx, double dt_s, const uint64_t* packets_per_box,
                            int* block_size, int* seg_per_iter, int* resort_interval,
                            int* reg_cap, int* tile, int* sort_curve);

/* ---- The exchange of a step split over several processes or GPUs.
   Packets are independent given the frozen absorbers (Sec. 2), so a step
   may be split by packet ids: every process holds a replica of the grid and
   traces a window of packet ids of every source (opts.pkt_begin/pkt_end,
   opts.chemistry = 0); the int64 deposits of all processes are summed (the
   one exchange of the step: Sec. 2's "reduction" strategy); then each
   process runs the per-cell update on the summed deposits.  Integer sums do
   not depend on their order, so the result is the same bits as one process
   tracing every packet, for any split.

   Device address of the deposits of box `box`: uint64[cells][4] (H I, He I,
   He II, heat) in the context's stream order; valid until crash_free.  A
   step's prep zeroes them; an in-place sum (e.g. an NCCL int64 all-reduce on
   crash_stream's stream, or after crash_sync) goes between the
   transport-only step and crash_chemistry.  n_cells may be NULL. */
crash_status crash_deposits_device(crash_ctx* ctx, int box, void** dev_ptr, int64_t* n_cells);
/* Host copies of the same array: read (int64[cells][4], synchronises) and
   overwrite (e.g. with the deposits summed over processes). */
crash_status crash_read_deposits(crash_ctx* ctx, int box, int64_t* host_out);
crash_status crash_write_deposits(crash_ctx* ctx, int box, const int64_t* host_in);
/* The per-cell update (Sec. 2; sub-sampled as in Sec. 3.2) of the last
   step, on the deposits the context now holds.  Only after a step run with
   opts.chemistry = 0, once, and with that step's dt_s (CRASH_ERR_STATE /
   CRASH_ERR_ARG otherwise).  Asynchronous on the context stream. */
crash_status crash_chemistry(crash_ctx* ctx, double dt_s);

crash_status crash_free(crash_ctx* ctx);
const char* crash_last_error(crash_ctx* ctx);   /* NULL ctx: last creation error */

/* ---- Transport without device allocation.
   The paper has no counterpart: this entry point exists for callers that
   cannot call cudaMalloc (code inside another framework's memory pool or
   under a fixed memory budget, plug-ins that may only use the buffers they
   are handed).  It runs the mixed-form transport of one grid for one step
   (emission, cell walk, attenuation, int64 deposition; no chemistry, no
   re-sort) exactly as crash_step does for a context with the same grid,
   sources and options, and allocates nothing: its scratch (packet queue of
   65536 packets per pass buffer, per-source tables for at most
   CRASH_NOALLOC_MAX_SOURCES sources, counters; about 21 MB) is a static
   device array that every GPU loading the library holds until the process
   exits.
     grid: host struct; nx, ny, nz, box_cm, he_over_h, isothermal, caseB and
       seed are used, the per-cell pointers are ignored; f_rec must be 0
       (source packets only: CRASH_ERR_ARG otherwise).
     pos_cells, ndot, bin_eV, bin_frac: host arrays as in crash_add_sources;
       1 <= n_src <= CRASH_NOALLOC_MAX_SOURCES (larger counts are rejected
       with CRASH_ERR_OVERFLOW), 1 <= n_bins <= 16.
     dt_s, step_index, packets_per_step: as in crash_step (step_index is the
       Philox step word); packets_per_step <= CRASH_NOALLOC_MAX_PACKETS
       (larger steps: CRASH_ERR_OVERFLOW); seg_per_pass: cells per wavefront
       pass (0 = 32).
     absorbers_dev: device float[nx*ny*nz][4] = n_HI, n_HeI, n_HeII, 0 (cm^-3),
       16-byte aligned (CRASH_ERR_ARG otherwise).
     deposits_dev: device uint64[nx*ny*nz][4] (HI, HeI, HeII, heat), 8-byte
       aligned (CRASH_ERR_ARG otherwise); the call ADDS its deposits, the
       caller zeroes the buffer for a fresh step.
     budget_out: host int64[8], laid out as CRASH_F_BUDGET, written.
     stream: a cudaStream_t (NULL: the default stream).
   The first call on a device looks up the scratch address with that device
   current (cudaGetSymbolAddress) and keeps it for the life of the process;
   make that first call before any stream capture.  A cudaDeviceReset in the
   caller's process invalidates the kept address: the call is unsupported
   after one.  The call synchronises `stream` before it returns.  Every call
   shares the one scratch array: calls that overlap on the GPU (from several
   host threads, or on several streams of one device) race and must not be
   issued.  Errors: CRASH_ERR_ARG / CRASH_ERR_OVERFLOW for rejected
   arguments (nothing is launched), CRASH_ERR_CUDA, CRASH_ERR_TIMEOUT for a
   device-side bound; crash_noalloc_last_error() gives the message. */
#define CRASH_NOALLOC_MAX_SOURCES 1024
#define CRASH_NOALLOC_MAX_PACKETS (1ull << 30)   /* 16384 queue chunks of 65536 packets */
crash_status crash_transport_noalloc(const crash_grid_desc* grid, int n_src, const double* pos_cells,
                                     const double* ndot, int n_bins, const double* bin_eV,
                                     const double* bin_frac, double dt_s, uint64_t step_index,
                                     uint64_t packets_per_step, int seg_per_pass,
                                     const float* absorbers_dev, unsigned long long* deposits_dev,
                                     int64_t* budget_out, void* stream);
const char* crash_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
