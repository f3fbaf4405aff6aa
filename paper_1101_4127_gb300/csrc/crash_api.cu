// crash_api.cu -- host runtime behind the C ABI of include/crash.h: context
// and device memory, source tables, the per-step launch sequence (optionally
// captured in a CUDA graph; NVTX ranges mark its phases), the diffuse
// recombination field's counts and re-emission, field I/O, checkpoints,
// event timing and the autotuner.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "crash_internal.cuh"

namespace {

// ionisation thresholds of H I, He I, He II (eV)
constexpr double kEth[3] = {13.6, 24.6, 54.4};
thread_local std::string g_create_error;

struct BoxHost {
  crash_grid_desc d;
  std::vector<double> pos, ndot, frac;   // sources of this box
  bool has_sources = false;
};

}  // namespace

struct crash_ctx {
  int n_boxes = 0;
  int precision = CRASH_FP64_PLAIN;
  std::vector<BoxHost> bh;
  std::vector<BoxMeta> meta;
  int64_t n_cells = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  // device buffers
  float* nH = nullptr;
  double *xHII = nullptr, *xHeII = nullptr, *xHeIII = nullptr, *T = nullptr;
  double* abs64 = nullptr;
  float* abs32 = nullptr;
  unsigned long long* dep = nullptr;
  BoxMeta* d_meta = nullptr;
  unsigned long long* budget = nullptr;
  unsigned long long* totals = nullptr;   // [n_boxes][8] running sums of the budget
  unsigned long long* step_dev = nullptr;
  unsigned long long* work = nullptr;
  int* err = nullptr;
  int* boxE = nullptr;
  double *src_pos = nullptr, *src_ndot = nullptr, *src_frac = nullptr;
  float* src_pos32 = nullptr;
  int* src_cell = nullptr;
  int64_t *src_base = nullptr, *src_rem = nullptr;
  int n_src_total = 0, src_cap = 0;
  // diffuse recombination field (some box has f_rec > 0)
  bool any_rec = false;
  double* rec = nullptr;            // [3][cells]
  long long* rec_list = nullptr;    // [cells][4]
  unsigned* rec_count = nullptr;
  unsigned long long* rec_rmax = nullptr;   // [n_boxes]
  double* snap_rec = nullptr;       // checkpoint copy of rec
  int rec_bin[3] = {-1, -1, -1};
  // bins
  int n_bins = 0;
  std::vector<double> bin_eV;
  BinTables tables{};
  // options / state
  crash_run_opts opts{};
  uint64_t step_host = 0;
  bool any_he = false, any_heat = false, any_periodic = false;
  std::string error;
  // exchange of a split step: the last step ran without chemistry and its
  // per-cell update is still due (crash_chemistry), with that step's dt
  bool chem_pending = false;
  double last_dt = 0.0;
  // timing
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  int ev_used = 0;
  double ms_accum = 0.0;
  int64_t launches_accum = 0;
  // graph of one step
  cudaGraphExec_t graph = nullptr;
  std::vector<uint64_t> graph_key;
  // mixed-form wavefront workspace
  void* wf = nullptr;
  int64_t launches = 0;          // kernels enqueued so far
  int64_t graph_launches = 0;    // kernels inside the captured step graph
  int max_iter = 0;              // largest per-box DDA bound
  double* snap = nullptr;        // checkpoint: 4 state fields
  unsigned long long* snap_step = nullptr;
  int64_t n_keys = 0;            // wavefront re-sort keys over all boxes
  int64_t n_tile_keys = 0;       // tile-pass keys over all boxes
  int max_tiles = 0;             // bound on the tiles one packet crosses
  int wf_mode = -1;              // wavefront option the workspace was sized for
  size_t bytes = 0;              // device bytes allocated by the context
};

// optional cap on the device memory a context may allocate (bytes; 0 = none)
static size_t memory_cap() {
  const char* v = getenv("CRASH_DEVICE_MEMORY_CAP");
  if (!v || !*v) return 0;
  return (size_t)strtoull(v, nullptr, 10);
}

static crash_status set_err(crash_ctx* c, crash_status st, const std::string& msg) {
  if (c) c->error = msg;
  else g_create_error = msg;
  return st;
}

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return set_err(c, e_ == cudaErrorMemoryAllocation ? CRASH_ERR_OOM : CRASH_ERR_CUDA, \
                     std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

extern "C" void crash_default_opts(crash_run_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->chemistry = 1;
  o->pkt_begin = 0;
  o->pkt_end = 0xFFFFFFFFu;
  o->chem_eps = 0.1;
  o->chem_max_sub = 10000;
  o->cool_mask = 63;
  o->block_size = 0;
  o->seg_per_iter = 0;
  o->resort_interval = 0;
  o->wavefront = 1;
  o->use_graph = 0;
  o->timing = 0;
  o->persistent = 1;
}

// ---------------------------------------------------------------- teardown
static void release(crash_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (auto& e : c->events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (c->wf) wavefront_destroy(c->wf);
  void* ptrs[] = {c->nH, c->xHII, c->xHeII, c->xHeIII, c->T, c->abs64, c->abs32, c->dep,
                  c->d_meta, c->budget, c->totals, c->step_dev, c->work, c->err, c->boxE, c->src_pos, c->src_ndot,
                  c->src_frac, c->src_base, c->src_rem, c->src_pos32, c->src_cell, c->snap,
                  c->snap_step, c->rec, c->rec_list, c->rec_count, c->rec_rmax, c->snap_rec};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" crash_status crash_free(crash_ctx* c) {
  if (!c) return CRASH_ERR_ARG;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  release(c);
  return CRASH_OK;
}

extern "C" const char* crash_last_error(crash_ctx* c) {
  return c ? c->error.c_str() : g_create_error.c_str();
}

extern "C" void* crash_stream(crash_ctx* c) { return c ? (void*)c->stream : nullptr; }

extern "C" int64_t crash_launch_count(crash_ctx* c) { return c ? c->launches : -1; }

// ---------------------------------------------------------------- creation
static crash_status validate_desc(const crash_grid_desc& d, int i) {
  crash_ctx* c = nullptr;
  char buf[160];
  if (d.nx < 1 || d.ny < 1 || d.nz < 1) {
    snprintf(buf, sizeof buf, "box %d: nx, ny, nz must be >= 1", i);
    return set_err(c, CRASH_ERR_ARG, buf);
  }
  if (!(d.box_cm > 0)) return set_err(c, CRASH_ERR_ARG, "box_cm must be positive");
  if (!(d.he_over_h >= 0)) return set_err(c, CRASH_ERR_ARG, "he_over_h must be >= 0");
  if (d.precision != CRASH_FP64_PLAIN && d.precision != CRASH_MIXED)
    return set_err(c, CRASH_ERR_ARG, "unknown precision");
  if ((int64_t)d.nx * d.ny * d.nz > ((int64_t)1 << 40))
    return set_err(c, CRASH_ERR_OVERFLOW, "grid too large");
  if (!d.T && !(d.T0 > 0)) return set_err(c, CRASH_ERR_ARG, "T0 must be positive");
  if (!(d.f_rec >= 0 && d.f_rec <= 1)) return set_err(c, CRASH_ERR_ARG, "f_rec must be in [0, 1]");
  if (d.coupling != 0 && d.coupling != 1) return set_err(c, CRASH_ERR_ARG, "coupling must be 0 or 1");
  if (d.periodic != 0 && d.periodic != 1) return set_err(c, CRASH_ERR_ARG, "periodic must be 0 or 1");
  for (int s = 0; s < 3; ++s)
    if (!(d.uv_rate[s] >= 0) || !std::isfinite(d.uv_rate[s]) || !(d.uv_heat_eV[s] >= 0) ||
        !std::isfinite(d.uv_heat_eV[s]))
      return set_err(c, CRASH_ERR_ARG, "uv_rate and uv_heat_eV must be finite and >= 0");
  return CRASH_OK;
}

static crash_status upload_box_state(crash_ctx* c, int b) {
  const crash_grid_desc& d = c->bh[b].d;
  const BoxMeta& m = c->meta[b];
  const size_t n = (size_t)m.ncell;
  std::vector<float> fh;
  std::vector<double> dh;
  if (d.n_H) {
    CK(cudaMemcpy(c->nH + m.cell_off, d.n_H, n * sizeof(float), cudaMemcpyHostToDevice));
  } else {
    fh.assign(n, (float)d.n_H0);
    CK(cudaMemcpy(c->nH + m.cell_off, fh.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  }
  const double* src[4] = {d.x_HII, d.x_HeII, d.x_HeIII, d.T};
  const double uni[4] = {d.x_HII0, d.x_HeII0, d.x_HeIII0, d.T0};
  double* dst[4] = {c->xHII, c->xHeII, c->xHeIII, c->T};
  for (int f = 0; f < 4; ++f) {
    if (src[f]) {
      CK(cudaMemcpy(dst[f] + m.cell_off, src[f], n * 8, cudaMemcpyHostToDevice));
    } else {
      dh.assign(n, uni[f]);
      CK(cudaMemcpy(dst[f] + m.cell_off, dh.data(), n * 8, cudaMemcpyHostToDevice));
    }
  }
  return CRASH_OK;
}

extern "C" crash_status crash_init_batch(int n_boxes, const crash_grid_desc* descs,
                                         crash_ctx** out) {
  crash_ctx* c = nullptr;
  if (!out) return set_err(c, CRASH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_boxes < 1 || n_boxes > CRASH_MAX_BOXES || !descs)
    return set_err(c, CRASH_ERR_ARG, "n_boxes must be in [1, 4096] with descriptors");
  for (int i = 0; i < n_boxes; ++i) {
    crash_status st = validate_desc(descs[i], i);
    if (st != CRASH_OK) return st;
    if (descs[i].precision != descs[0].precision)
      return set_err(c, CRASH_ERR_ARG, "all boxes of a batch need the same precision");
  }
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
    return set_err(c, CRASH_ERR_CUDA, "no CUDA device available");
  cudaGetDevice(&dev);
  c = new crash_ctx();
  c->device = dev;
  c->n_boxes = n_boxes;
  c->precision = descs[0].precision;
  c->bh.resize(n_boxes);
  c->meta.resize(n_boxes);
  crash_default_opts(&c->opts);
  int64_t off = 0;
  for (int i = 0; i < n_boxes; ++i) {
    const crash_grid_desc& d = descs[i];
    c->bh[i].d = d;
    BoxMeta& m = c->meta[i];
    memset(&m, 0, sizeof m);
    m.nx = d.nx; m.ny = d.ny; m.nz = d.nz;
    m.isothermal = d.isothermal ? 1 : 0;
    m.cell_off = off;
    m.ncell = (int64_t)d.nx * d.ny * d.nz;
    m.dl = d.box_cm / d.nx;
    m.dlf = (float)m.dl;
    m.he = d.he_over_h;
    m.T_cmb = d.z_compton >= 0 ? 2.725 * (1.0 + d.z_compton) : 0.0;
    m.seed = d.seed;
    m.caseB = d.caseB ? 1 : 0;
    m.max_iter = d.nx + d.ny + d.nz + 3;
    m.f_rec = d.f_rec;
    m.coupling = d.coupling;
    m.periodic = d.periodic;
    for (int s = 0; s < 3; ++s) {
      m.uv[s] = d.uv_rate[s];
      m.uve[s] = d.uv_heat_eV[s];
    }
    c->any_rec |= d.f_rec > 0;
    c->any_periodic |= d.periodic != 0;
    off += m.ncell;
    c->any_he |= d.he_over_h > 0;
    c->any_heat |= !d.isothermal;
  }
  c->n_cells = off;
  // wavefront sort keys: per box, Morton order of 8^3-cell buckets times 8 octants
  int64_t keys = 0;
  for (int i = 0; i < n_boxes; ++i) {
    BoxMeta& m = c->meta[i];
    int cmax = std::max(std::max((m.nx + 7) / 8, (m.ny + 7) / 8), (m.nz + 7) / 8);
    int bits = 0;
    while ((1 << bits) < cmax) ++bits;
    m.bucket_bits = bits;
    m.bucket_off = keys;
    keys += (int64_t)8 << (3 * bits);
    c->max_iter = std::max(c->max_iter, m.max_iter);
  }
  c->n_keys = keys;
  // tile-pass keys: 16^3-cell tiles times 8 octants (fewer than the 8^3 keys)
  int64_t tkeys = 0;
  for (int i = 0; i < n_boxes; ++i) {
    BoxMeta& m = c->meta[i];
    int cmax = std::max(std::max((m.nx + 15) / 16, (m.ny + 15) / 16), (m.nz + 15) / 16);
    int bits = 0;
    while ((1 << bits) < cmax) ++bits;
    m.tile_bits = bits;
    m.tile_off = tkeys;
    tkeys += (int64_t)8 << (3 * bits);
    c->max_tiles = std::max(c->max_tiles, (m.nx + 15) / 16 + (m.ny + 15) / 16 + (m.nz + 15) / 16 + 3);
  }
  c->n_tile_keys = tkeys;
  auto fail = [&](crash_status st) { release(c); return st; };
  if (c->precision == CRASH_MIXED) {
    if (n_boxes > 2048) {
      g_create_error = "mixed form: at most 2048 boxes per batch";
      return fail(CRASH_ERR_OVERFLOW);
    }
    for (int i = 0; i < n_boxes; ++i)
      if (descs[i].nx > 65535 || descs[i].ny > 65535 || descs[i].nz > 65535 ||
          (int64_t)descs[i].nx * descs[i].ny * descs[i].nz >= ((int64_t)1 << 31)) {
        g_create_error = "mixed form: each axis <= 65535 cells and < 2^31 cells per box";
        return fail(CRASH_ERR_OVERFLOW);
      }
    if (keys > (int64_t)4096 * 1024) {
      g_create_error = "mixed form: too many boxes/cells for the re-sort key space";
      return fail(CRASH_ERR_OVERFLOW);
    }
  }
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { g_create_error = cudaGetErrorString(e); return fail(CRASH_ERR_CUDA); }
  const size_t n = (size_t)c->n_cells;
  struct A { void** p; size_t bytes; };
  std::vector<A> allocs = {
      {(void**)&c->nH, n * 4}, {(void**)&c->xHII, n * 8}, {(void**)&c->xHeII, n * 8},
      {(void**)&c->xHeIII, n * 8}, {(void**)&c->T, n * 8}, {(void**)&c->dep, n * 32},
      {(void**)&c->d_meta, sizeof(BoxMeta) * n_boxes},
      {(void**)&c->budget, 64 * (size_t)n_boxes}, {(void**)&c->totals, 64 * (size_t)n_boxes},
      {(void**)&c->step_dev, 8}, {(void**)&c->work, 8},
      {(void**)&c->err, sizeof(int)}, {(void**)&c->boxE, sizeof(int) * n_boxes}};
  if (c->precision == CRASH_MIXED) allocs.push_back({(void**)&c->abs32, n * 16});
  else allocs.push_back({(void**)&c->abs64, n * 32});
  if (c->any_rec) {
    allocs.push_back({(void**)&c->rec, n * 24});
    allocs.push_back({(void**)&c->rec_list, n * 32});
    allocs.push_back({(void**)&c->rec_count, 16});
    allocs.push_back({(void**)&c->rec_rmax, 8 * (size_t)n_boxes});
  }
  {
    size_t want = 0;
    for (auto& a : allocs) want += a.bytes;
    const size_t cap = memory_cap();
    if (cap && want > cap) {
      g_create_error = "device memory cap (CRASH_DEVICE_MEMORY_CAP) exceeded: need " +
                       std::to_string(want) + " bytes";
      return fail(CRASH_ERR_OOM);
    }
    c->bytes = want;
  }
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      g_create_error = std::string("device allocation failed: ") + cudaGetErrorString(e);
      return fail(e == cudaErrorMemoryAllocation ? CRASH_ERR_OOM : CRASH_ERR_CUDA);
    }
  }
  cudaMemset(c->budget, 0, 64 * (size_t)n_boxes);
  cudaMemset(c->totals, 0, 64 * (size_t)n_boxes);
  cudaMemset(c->step_dev, 0, 8);
  cudaMemset(c->err, 0, sizeof(int));
  cudaMemset(c->dep, 0, n * 32);
  if (c->any_rec) cudaMemset(c->rec, 0, n * 24);
  for (int i = 0; i < n_boxes; ++i) {
    crash_status st = upload_box_state(c, i);
    if (st != CRASH_OK) {
      g_create_error = c->error;
      return fail(st);
    }
  }
  *out = c;
  return CRASH_OK;
}

extern "C" crash_status crash_init_grid(const crash_grid_desc* d, crash_ctx** out) {
  if (!d) return set_err(nullptr, CRASH_ERR_ARG, "desc is NULL");
  return crash_init_batch(1, d, out);
}

// ---------------------------------------------------------------- sources
void cross_sections(int nb, const double* E, BinTables& t, int& heatF) {
  double emax = 0.0;
  for (int j = 0; j < nb; ++j) {
    const double e = E[j];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    // hydrogenic H I and He II: sigma_0 (E_th / E)^3
    if (e >= kEth[0]) { const double r = kEth[0] / e; s0 = 6.30e-18 * ((r * r) * r); }
    if (e >= kEth[2]) { const double r = kEth[2] / e; s2 = 1.58e-18 * ((r * r) * r); }
    // He I: Osterbrock (1989) fit with beta = 1.66, s = 2.05
    if (e >= kEth[1]) {
      const double y = e / kEth[1];
      s1 = 7.83e-18 * (1.66 * pow(y, -2.05) + (1.0 - 1.66) * pow(y, -3.05));
    }
    t.sigma[0][j] = s0; t.sigma[1][j] = s1; t.sigma[2][j] = s2;
    for (int s = 0; s < 3; ++s)
      if (e >= kEth[s] && e - kEth[s] > emax) emax = e - kEth[s];
  }
  heatF = 0;
  if (emax > 1.0) {
    int ex;
    double m = frexp(emax, &ex);
    heatF = (m == 0.5) ? ex - 1 : ex;
  }
  for (int s = 0; s < 3; ++s)
    for (int j = 0; j < nb; ++j) {
      t.wheat[s][j] = E[j] >= kEth[s] ? ldexp(E[j] - kEth[s], -heatF) : 0.0;
      t.sigma32[s][j] = (float)t.sigma[s][j];
      t.wheat32[s][j] = (float)t.wheat[s][j];
      t.sw32[s][j] = t.sigma32[s][j] * t.wheat32[s][j];
    }
  for (int s = 0; s < 3; ++s) {
    t.sigma32_max[s] = 0.f;
    for (int j = 0; j < nb; ++j) t.sigma32_max[s] = std::max(t.sigma32_max[s], t.sigma32[s][j]);
  }
  t.n_bins = nb;
}

static crash_status rebuild_sources(crash_ctx* c) {
  int total = 0;
  for (int b = 0; b < c->n_boxes; ++b) {
    c->meta[b].src_off = total;
    c->meta[b].n_src = (int)c->bh[b].ndot.size();
    total += c->meta[b].n_src;
  }
  const int nb = c->n_bins;
  if (total > c->src_cap) {
    void* old[] = {c->src_pos, c->src_ndot, c->src_frac, c->src_base, c->src_rem, c->src_pos32,
                   c->src_cell};
    for (void* p : old)
      if (p) cudaFree(p);
    c->src_pos = c->src_ndot = c->src_frac = nullptr;
    c->src_base = c->src_rem = nullptr;
    c->src_pos32 = nullptr;
    c->src_cell = nullptr;
    CK(cudaMalloc(&c->src_pos32, sizeof(float) * 3 * total));
    CK(cudaMalloc(&c->src_cell, sizeof(int) * 3 * total));
    CK(cudaMalloc(&c->src_pos, sizeof(double) * 3 * total));
    CK(cudaMalloc(&c->src_ndot, sizeof(double) * total));
    CK(cudaMalloc(&c->src_frac, sizeof(double) * total * CRASH_MAX_BINS));
    CK(cudaMalloc(&c->src_base, sizeof(int64_t) * total * CRASH_MAX_BINS));
    CK(cudaMalloc(&c->src_rem, sizeof(int64_t) * total * CRASH_MAX_BINS));
    c->src_cap = total;
  }
  std::vector<double> pos, ndot, frac;
  pos.reserve(3 * total); ndot.reserve(total); frac.reserve((size_t)total * nb);
  for (int b = 0; b < c->n_boxes; ++b) {
    const BoxHost& h = c->bh[b];
    pos.insert(pos.end(), h.pos.begin(), h.pos.end());
    ndot.insert(ndot.end(), h.ndot.begin(), h.ndot.end());
    frac.insert(frac.end(), h.frac.begin(), h.frac.end());
  }
  c->n_src_total = total;
  if (total) {
    std::vector<float> pos32(pos.size());
    std::vector<int> cell(pos.size());
    for (size_t i = 0; i < pos.size(); ++i) {
      pos32[i] = (float)pos[i];
      cell[i] = (int)floor(pos[i]);
    }
    CK(cudaMemcpy(c->src_pos32, pos32.data(), pos32.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->src_cell, cell.data(), cell.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->src_pos, pos.data(), pos.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->src_ndot, ndot.data(), ndot.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->src_frac, frac.data(), frac.size() * 8, cudaMemcpyHostToDevice));
  }
  return CRASH_OK;
}

extern "C" crash_status crash_add_sources_box(crash_ctx* c, int box, int n_src,
                                              const double* pos, const double* ndot,
                                              int n_bins, const double* bin_eV,
                                              const double* bin_frac) {
  if (!c) return CRASH_ERR_ARG;
  if (box < 0 || box >= c->n_boxes) return set_err(c, CRASH_ERR_ARG, "box index out of range");
  if (n_src < 1 || !pos || !ndot || !bin_eV || !bin_frac)
    return set_err(c, CRASH_ERR_ARG, "need n_src >= 1 and non-NULL arrays");
  if (n_bins < 1 || n_bins > CRASH_MAX_BINS)
    return set_err(c, CRASH_ERR_OVERFLOW, "n_bins must be in [1, 16]");
  for (int j = 0; j < n_bins; ++j)
    if (!(bin_eV[j] > 0)) return set_err(c, CRASH_ERR_ARG, "bin energies must be positive");
  // all boxes share one bin table
  bool others = false;
  for (int b = 0; b < c->n_boxes; ++b) others |= (b != box && c->bh[b].has_sources);
  if (others && (n_bins != c->n_bins || !std::equal(bin_eV, bin_eV + n_bins, c->bin_eV.begin())))
    return set_err(c, CRASH_ERR_ARG, "all boxes must use the same frequency bins");
  const crash_grid_desc& d = c->bh[box].d;
  for (int s = 0; s < n_src; ++s) {
    const double* p = pos + 3 * s;
    if (!(p[0] >= 0 && p[0] < d.nx && p[1] >= 0 && p[1] < d.ny && p[2] >= 0 && p[2] < d.nz))
      return set_err(c, CRASH_ERR_ARG, "source position outside the grid");
    if (!(ndot[s] >= 0) || !isfinite(ndot[s]))
      return set_err(c, CRASH_ERR_ARG, "source rates must be finite and >= 0");
    for (int j = 0; j < n_bins; ++j)
      if (!(bin_frac[(size_t)s * n_bins + j] >= 0))
        return set_err(c, CRASH_ERR_ARG, "bin fractions must be >= 0");
  }
  BoxHost& h = c->bh[box];
  h.pos.assign(pos, pos + 3 * n_src);
  h.ndot.assign(ndot, ndot + n_src);
  h.frac.assign(bin_frac, bin_frac + (size_t)n_src * n_bins);
  h.has_sources = true;
  c->n_bins = n_bins;
  c->bin_eV.assign(bin_eV, bin_eV + n_bins);
  int heatF = 0;
  cross_sections(n_bins, bin_eV, c->tables, heatF);
  // re-emitted photons of H I, He I, He II: the lowest bin at or above the
  // species' ionisation threshold (-1 when there is none)
  const double Eth[3] = {13.6, 24.6, 54.4};
  for (int sp = 0; sp < 3; ++sp) {
    c->rec_bin[sp] = -1;
    for (int j = 0; j < n_bins; ++j)
      if (bin_eV[j] >= Eth[sp] && (c->rec_bin[sp] < 0 || bin_eV[j] < bin_eV[c->rec_bin[sp]]))
        c->rec_bin[sp] = j;
  }
  for (int b = 0; b < c->n_boxes; ++b) c->meta[b].heatF = heatF;
  double sum = 0.0;                       // in source order, as the specification sums
  for (int s = 0; s < n_src; ++s) sum += ndot[s];
  c->meta[box].ndot_sum = sum;
  crash_status st = rebuild_sources(c);
  if (st != CRASH_OK) return st;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return CRASH_OK;
}

extern "C" crash_status crash_add_sources(crash_ctx* c, int n_src, const double* pos,
                                          const double* ndot, int n_bins, const double* bin_eV,
                                          const double* bin_frac) {
  return crash_add_sources_box(c, 0, n_src, pos, ndot, n_bins, bin_eV, bin_frac);
}

extern "C" crash_status crash_set_options(crash_ctx* c, const crash_run_opts* o) {
  if (!c || !o) return set_err(c, CRASH_ERR_ARG, "NULL argument");
  if (o->pkt_end < o->pkt_begin) return set_err(c, CRASH_ERR_ARG, "pkt_end < pkt_begin");
  if (!(o->chem_eps > 0) || o->chem_max_sub < 1)
    return set_err(c, CRASH_ERR_ARG, "chem_eps must be > 0 and chem_max_sub >= 1");
  if (o->block_size < 0 || o->block_size > 1024 || (o->block_size % 32))
    return set_err(c, CRASH_ERR_ARG, "block_size must be a multiple of 32 in [0, 1024]");
  if (o->seg_per_iter < 0) return set_err(c, CRASH_ERR_ARG, "seg_per_iter must be >= 0");
  if (o->chunk_packets < 0) return set_err(c, CRASH_ERR_ARG, "chunk_packets must be >= 0");
  c->opts = *o;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return CRASH_OK;
}

extern "C" crash_status crash_get_options(crash_ctx* c, crash_run_opts* o) {
  if (!c || !o) return set_err(c, CRASH_ERR_ARG, "NULL argument");
  *o = c->opts;
  return CRASH_OK;
}

extern "C" crash_status crash_checkpoint(crash_ctx* c, int op) {
  if (!c) return CRASH_ERR_ARG;
  cudaSetDevice(c->device);
  const size_t n = (size_t)c->n_cells;
  double* f[4] = {c->xHII, c->xHeII, c->xHeIII, c->T};
  if (op == CRASH_CKPT_SAVE) {
    if (!c->snap) {
      CK(cudaMalloc(&c->snap, n * 8 * 4));
      CK(cudaMalloc(&c->snap_step, 8));
    }
    for (int i = 0; i < 4; ++i)
      CK(cudaMemcpyAsync(c->snap + i * n, f[i], n * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->snap_step, c->step_dev, 8, cudaMemcpyDeviceToDevice, c->stream));
    if (c->any_rec) {
      if (!c->snap_rec) CK(cudaMalloc(&c->snap_rec, n * 24));
      CK(cudaMemcpyAsync(c->snap_rec, c->rec, n * 24, cudaMemcpyDeviceToDevice, c->stream));
    }
    return CRASH_OK;
  }
  if (op != CRASH_CKPT_RESTORE_STATE && op != CRASH_CKPT_RESTORE)
    return set_err(c, CRASH_ERR_ARG, "unknown checkpoint op");
  if (!c->snap) return set_err(c, CRASH_ERR_STATE, "no checkpoint saved");
  for (int i = 0; i < 4; ++i)
    CK(cudaMemcpyAsync(f[i], c->snap + i * n, n * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (c->any_rec && c->snap_rec)
    CK(cudaMemcpyAsync(c->rec, c->snap_rec, n * 24, cudaMemcpyDeviceToDevice, c->stream));
  if (op == CRASH_CKPT_RESTORE)
    CK(cudaMemcpyAsync(c->step_dev, c->snap_step, 8, cudaMemcpyDeviceToDevice, c->stream));
  return CRASH_OK;
}

extern "C" crash_status crash_set_step_index(crash_ctx* c, uint64_t step) {
  if (!c) return CRASH_ERR_ARG;
  cudaSetDevice(c->device);
  unsigned long long v = step;
  CK(cudaMemcpyAsync(c->step_dev, &v, 8, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->step_host = step;
  return CRASH_OK;
}

// ---------------------------------------------------------------- step
// end of step: advance the step index and add the step's budget to the totals
__global__ void k_end_step(unsigned long long* s, const unsigned long long* budget,
                           unsigned long long* totals, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *s += 1ull;
  if (i < 8 * n) {
    int k = i & 7;
    if (k == 5 || k == 6) totals[i] = budget[i];
    else totals[i] += budget[i];
  }
}

static StepArgs make_args(crash_ctx* c, double dt, int64_t total) {
  StepArgs a;
  memset(&a, 0, sizeof a);
  a.boxes = c->d_meta;
  a.n_boxes = c->n_boxes;
  a.step_dev = c->step_dev;
  a.dt = dt;
  a.total_packets = total;
  a.src_pos = c->src_pos; a.src_ndot = c->src_ndot; a.src_frac = c->src_frac;
  a.src_pos32 = c->src_pos32; a.src_cell = c->src_cell;
  a.src_base = c->src_base; a.src_rem = c->src_rem;
  a.box_E = c->boxE;
  a.n_src_total = c->n_src_total;
  a.nH = c->nH; a.xHII = c->xHII; a.xHeII = c->xHeII; a.xHeIII = c->xHeIII; a.T = c->T;
  a.abs64 = c->abs64; a.abs32 = c->abs32; a.dep = c->dep;
  a.n_cells_total = c->n_cells;
  a.budget = c->budget;
  a.work = c->work;
  a.n_tile_keys = c->n_tile_keys;
  a.max_tiles = c->max_tiles;
  a.err = c->err;
  a.any_he = c->any_he; a.any_heat = c->any_heat;
  a.any_periodic = c->any_periodic;
  a.max_iter_step = c->max_iter;
  a.chemistry = c->opts.chemistry;
  a.fp32_rates = c->precision == CRASH_MIXED;
  a.chem_eps = c->opts.chem_eps;
  a.chem_max_sub = c->opts.chem_max_sub;
  a.cool_mask = c->opts.cool_mask;
  a.any_rec = c->any_rec ? 1 : 0;
  a.rec = c->rec;
  a.rec_list = c->rec_list;
  a.rec_count = c->rec_count;
  a.rec_rmax = c->rec_rmax;
  for (int sp = 0; sp < 3; ++sp) a.rec_bin[sp] = c->rec_bin[sp];
  return a;
}

// NVTX range over a phase of the host-side launch sequence, so that a
// profiler can select the kernels of one phase (ncu --nvtx --nvtx-include);
// without a profiler attached a range costs a few nanoseconds
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// the launch sequence of one step (everything on c->stream)
static crash_status enqueue_step(crash_ctx* c, const StepArgs& a, bool timing, int64_t* nk) {
  NvtxRange step_range("crash step");
  CK(cudaMemsetAsync(c->budget, 0, 64 * (size_t)c->n_boxes, c->stream));
  launch_prep(a, c->precision, c->stream);
  if (c->any_rec) launch_rec_max(a, c->stream);      // the quantum covers the re-emission
  launch_budget(a, c->tables, c->stream);
  *nk = 3 + (c->opts.chemistry ? 1 : 0);   // prep, budget, end-of-step, chemistry
  // diffuse recombination field: this step's re-emitting cells (from the
  // counts of earlier steps), traced after the source packets
  if (c->any_rec) {
    launch_rec_select(a, c->stream);
    *nk += 2;
  }
  {
    NvtxRange transport_range("transport");
    if (c->precision == CRASH_MIXED) {
      // tile passes key packets by the Morton index of their 16^3 tile, which
      // the tile kernel decodes back into the tile's position: the Hilbert
      // option applies to the bucket keys of the other passes only
      crash_run_opts o = c->opts;
      if (o.tile) o.sort_curve = 0;
      int rc = launch_trace_mixed(a, c->tables, o, c->wf, a.max_iter_step, c->stream,
                                  timing ? &c->events : nullptr, &c->ev_used);
      if (rc < 0) return set_err(c, CRASH_ERR_CUDA, "mixed transport launch failed");
      *nk += rc;
    } else {
      *nk += 1;
      if (timing) {
        if (c->ev_used >= (int)c->events.size()) {
          cudaEvent_t e0, e1;
          CK(cudaEventCreate(&e0));
          CK(cudaEventCreate(&e1));
          c->events.push_back({e0, e1});
        }
        CK(cudaEventRecord(c->events[c->ev_used].first, c->stream));
      }
      launch_trace_fp64(a, c->tables, c->opts.block_size, c->stream);
      if (timing) {
        CK(cudaEventRecord(c->events[c->ev_used].second, c->stream));
        c->ev_used++;
      }
    }
    if (c->any_rec) {
      if (c->precision == CRASH_MIXED) {
        if (launch_rec_mixed(a, c->tables, c->stream) < 0)
          return set_err(c, CRASH_ERR_CUDA, "re-emission launch failed");
      } else {
        launch_rec_fp64(a, c->tables, c->stream);
      }
      *nk += 1;
    }
  }   // transport range
  if (c->opts.chemistry) {
    NvtxRange chem_range("chemistry");
    launch_chemistry(a, c->stream);
  }
  k_end_step<<<(8 * c->n_boxes + 255) / 256, 256, 0, c->stream>>>(c->step_dev, c->budget,
                                                                    c->totals, c->n_boxes);
  CK(cudaGetLastError());
  return CRASH_OK;
}

extern "C" crash_status crash_step_batch(crash_ctx* c, double dt, const uint64_t* P) {
  if (!c) return CRASH_ERR_ARG;
  if (!(dt > 0) || !isfinite(dt)) return set_err(c, CRASH_ERR_ARG, "dt must be positive");
  if (!P) return set_err(c, CRASH_ERR_ARG, "packets_per_box is NULL");
  cudaSetDevice(c->device);
  int64_t total = 0;
  std::vector<uint64_t> key = {(uint64_t)c->n_boxes};
  {
    uint64_t dtb;
    memcpy(&dtb, &dt, 8);
    key.push_back(dtb);
  }
  for (int b = 0; b < c->n_boxes; ++b) {
    if (!c->bh[b].has_sources) return set_err(c, CRASH_ERR_STATE, "a box has no sources");
    BoxMeta& m = c->meta[b];
    if (P[b] == 0 || P[b] % (uint64_t)m.n_src)
      return set_err(c, CRASH_ERR_ARG, "packets_per_step must be a positive multiple of n_src");
    const uint64_t Ns = P[b] / (uint64_t)m.n_src;
    if (Ns > 0xFFFFFFFFull) return set_err(c, CRASH_ERR_OVERFLOW, "more than 2^32-1 packets per source");
    m.pkts_per_src = Ns;
    m.win_lo = (uint32_t)std::min<uint64_t>(c->opts.pkt_begin, Ns);
    m.win_hi = (uint32_t)std::min<uint64_t>(c->opts.pkt_end, Ns);
    if (m.win_hi < m.win_lo) m.win_hi = m.win_lo;
    m.pkt_off = total;
    m.pkt_count = (int64_t)m.n_src * (int64_t)(m.win_hi - m.win_lo);
    total += m.pkt_count;
    key.push_back(P[b]);
  }
  if (total > ((int64_t)1 << 40)) return set_err(c, CRASH_ERR_OVERFLOW, "too many packets in one step");
  // DDA bound of this step: a periodic box's packets travel c dt, so their
  // walks are bounded by 2 L + 4 face crossings (L = c dt / dl cells)
  int step_max_iter = c->max_iter;
  for (int b = 0; b < c->n_boxes; ++b) {
    BoxMeta& m = c->meta[b];
    if (!m.periodic) continue;
    const double L = (CRASH_C_LIGHT * dt) / m.dl;
    if (!(L <= 536870912.0))
      return set_err(c, CRASH_ERR_ARG, "periodic box: c dt exceeds 2^29 cells");
    m.max_iter = (int)(2.0 * L) + 4;
    m.path_cells32 = (float)L;
    step_max_iter = std::max(step_max_iter, m.max_iter);
    key.push_back((uint64_t)m.max_iter);
  }
  CK(cudaMemcpyAsync(c->d_meta, c->meta.data(), sizeof(BoxMeta) * c->n_boxes,
                     cudaMemcpyHostToDevice, c->stream));
  if (c->precision == CRASH_MIXED) {
    // packet queue: sized to the step (at most 2^28 packets per chunk, 38 GB
    // with 8 bins); none when every packet is traced to the end by its own
    // thread.  Larger chunks put more packets in each sort bucket of a pass,
    // so more crossings of a cell fall close together in time and its
    // deposit record is reused in L2.
    const int64_t chunk = c->opts.chunk_packets > 0 ? (int64_t)c->opts.chunk_packets : (int64_t)1 << 28;
    const int64_t want = (c->opts.wavefront && !c->any_periodic) ? std::min<int64_t>(total, chunk) : 0;
    if (c->wf && (c->wf_mode != c->opts.wavefront || wavefront_capacity(c->wf) < want)) {
      CK(cudaStreamSynchronize(c->stream));
      wavefront_destroy(c->wf);
      c->wf = nullptr;
      if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    }
    if (!c->wf) {
      const size_t cap = memory_cap();
      const size_t need = (size_t)want * (size_t)(2 * (((32 + 4 * c->n_bins) + 15) / 16 * 16) + 12);
      if (cap && c->bytes + need > cap)
        return set_err(c, CRASH_ERR_OOM, "device memory cap (CRASH_DEVICE_MEMORY_CAP) exceeded by the packet queue");
      cudaError_t e = cudaSuccess;
      c->wf = wavefront_create(want, c->n_keys, c->n_bins, &e);
      if (!c->wf) return set_err(c, CRASH_ERR_OOM, std::string("wavefront workspace: ") + cudaGetErrorString(e));
      c->wf_mode = c->opts.wavefront;
    }
  }
  StepArgs a = make_args(c, dt, total);
  a.max_iter_step = step_max_iter;
  const bool timing = c->opts.timing != 0;
  crash_status st;
  if (c->opts.use_graph && !timing) {
    if (!c->graph || c->graph_key != key) {
      if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      st = enqueue_step(c, a, false, &c->graph_launches);
      cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      if (st != CRASH_OK) return st;
      if (e != cudaSuccess) return set_err(c, CRASH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return set_err(c, CRASH_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      c->graph_key = key;
    }
    CK(cudaGraphLaunch(c->graph, c->stream));
    c->launches += c->graph_launches;
  } else {
    int64_t nk = 0;
    st = enqueue_step(c, a, timing, &nk);
    if (st != CRASH_OK) return st;
    c->launches += nk;
  }
  c->step_host += 1;
  c->chem_pending = !c->opts.chemistry;
  c->last_dt = dt;
  return CRASH_OK;
}

extern "C" crash_status crash_step(crash_ctx* c, double dt, uint64_t P) {
  if (!c) return CRASH_ERR_ARG;
  if (c->n_boxes != 1) return set_err(c, CRASH_ERR_ARG, "batched context: use crash_step_batch");
  return crash_step_batch(c, dt, &P);
}

static crash_status check_device_error(crash_ctx* c) {
  int e = 0;
  CK(cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    std::string m = "device-side limit hit:";
    if (e & ERR_DDA_LIMIT) m += " DDA iteration limit;";
    if (e & ERR_DIRECTION) m += " direction sampling exceeded 64 attempts;";
    if (e & ERR_QUEUE) m += " packet queue overflow;";
    if (e & ERR_WATCHDOG) m += " wavefront pass limit;";
    return set_err(c, CRASH_ERR_TIMEOUT, m);
  }
  return CRASH_OK;
}

extern "C" crash_status crash_sync(crash_ctx* c) {
  if (!c) return CRASH_ERR_ARG;
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

// ---------------------------------------------------------------- fields
extern "C" crash_status crash_read_fields_box(crash_ctx* c, int box, int f, void* out) {
  if (!c) return CRASH_ERR_ARG;
  if (!out) return set_err(c, CRASH_ERR_ARG, "output is NULL");
  if (box < 0 || box >= c->n_boxes) return set_err(c, CRASH_ERR_ARG, "box index out of range");
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));
  crash_status st = check_device_error(c);
  if (st != CRASH_OK) return st;
  const BoxMeta& m = c->meta[box];
  const size_t n = (size_t)m.ncell;
  switch (f) {
    case CRASH_F_XHII: CK(cudaMemcpy(out, c->xHII + m.cell_off, n * 8, cudaMemcpyDeviceToHost)); break;
    case CRASH_F_XHEII: CK(cudaMemcpy(out, c->xHeII + m.cell_off, n * 8, cudaMemcpyDeviceToHost)); break;
    case CRASH_F_XHEIII: CK(cudaMemcpy(out, c->xHeIII + m.cell_off, n * 8, cudaMemcpyDeviceToHost)); break;
    case CRASH_F_T: CK(cudaMemcpy(out, c->T + m.cell_off, n * 8, cudaMemcpyDeviceToHost)); break;
    case CRASH_F_DEP_HI: case CRASH_F_DEP_HEI: case CRASH_F_DEP_HEII: case CRASH_F_DEP_E:
      CK(cudaMemcpy2D(out, 8, c->dep + 4 * m.cell_off + (f - CRASH_F_DEP_HI), 32, 8, n,
                      cudaMemcpyDeviceToHost));
      break;
    case CRASH_F_BUDGET: CK(cudaMemcpy(out, c->budget + 8 * box, 64, cudaMemcpyDeviceToHost)); break;
    case CRASH_F_TOTALS: CK(cudaMemcpy(out, c->totals + 8 * box, 64, cudaMemcpyDeviceToHost)); break;
    case CRASH_F_REC_HI: case CRASH_F_REC_HEI: case CRASH_F_REC_HEII:
      if (!c->rec) return set_err(c, CRASH_ERR_STATE, "the diffuse recombination field is off (f_rec = 0)");
      CK(cudaMemcpy(out, c->rec + (size_t)(f - CRASH_F_REC_HI) * c->n_cells + m.cell_off, n * 8,
                    cudaMemcpyDeviceToHost));
      break;
    case CRASH_F_NH: {
      std::vector<float> tmp(n);
      CK(cudaMemcpy(tmp.data(), c->nH + m.cell_off, n * 4, cudaMemcpyDeviceToHost));
      double* o = (double*)out;
      for (size_t i = 0; i < n; ++i) o[i] = (double)tmp[i];
      break;
    }
    default: return set_err(c, CRASH_ERR_ARG, "unknown field id");
  }
  return CRASH_OK;
}

extern "C" crash_status crash_read_fields(crash_ctx* c, int f, void* out) {
  return crash_read_fields_box(c, 0, f, out);
}

extern "C" crash_status crash_write_fields_box(crash_ctx* c, int box, int f, const void* in) {
  if (!c) return CRASH_ERR_ARG;
  if (!in) return set_err(c, CRASH_ERR_ARG, "input is NULL");
  if (box < 0 || box >= c->n_boxes) return set_err(c, CRASH_ERR_ARG, "box index out of range");
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));
  const BoxMeta& m = c->meta[box];
  const size_t n = (size_t)m.ncell;
  double* dst = nullptr;
  switch (f) {
    case CRASH_F_XHII: dst = c->xHII; break;
    case CRASH_F_XHEII: dst = c->xHeII; break;
    case CRASH_F_XHEIII: dst = c->xHeIII; break;
    case CRASH_F_T: dst = c->T; break;
    case CRASH_F_REC_HI: case CRASH_F_REC_HEI: case CRASH_F_REC_HEII:
      if (!c->rec) return set_err(c, CRASH_ERR_STATE, "the diffuse recombination field is off (f_rec = 0)");
      dst = c->rec + (size_t)(f - CRASH_F_REC_HI) * c->n_cells;
      break;
    default: return set_err(c, CRASH_ERR_ARG, "field is not writable");
  }
  CK(cudaMemcpy(dst + m.cell_off, in, n * 8, cudaMemcpyHostToDevice));
  return CRASH_OK;
}

extern "C" crash_status crash_write_fields(crash_ctx* c, int f, const void* in) {
  return crash_write_fields_box(c, 0, f, in);
}

// ---------------------------------------------------------------- exchange
extern "C" crash_status crash_deposits_device(crash_ctx* c, int box, void** dev_ptr, int64_t* n_cells) {
  if (!c) return CRASH_ERR_ARG;
  if (!dev_ptr) return set_err(c, CRASH_ERR_ARG, "dev_ptr is NULL");
  if (box < 0 || box >= c->n_boxes) return set_err(c, CRASH_ERR_ARG, "box index out of range");
  *dev_ptr = (void*)(c->dep + 4 * c->meta[box].cell_off);
  if (n_cells) *n_cells = c->meta[box].ncell;
  return CRASH_OK;
}

extern "C" crash_status crash_read_deposits(crash_ctx* c, int box, int64_t* out) {
  if (!c) return CRASH_ERR_ARG;
  if (!out) return set_err(c, CRASH_ERR_ARG, "output is NULL");
  if (box < 0 || box >= c->n_boxes) return set_err(c, CRASH_ERR_ARG, "box index out of range");
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));
  crash_status st = check_device_error(c);
  if (st != CRASH_OK) return st;
  const BoxMeta& m = c->meta[box];
  CK(cudaMemcpy(out, c->dep + 4 * m.cell_off, (size_t)m.ncell * 32, cudaMemcpyDeviceToHost));
  return CRASH_OK;
}

extern "C" crash_status crash_write_deposits(crash_ctx* c, int box, const int64_t* in) {
  if (!c) return CRASH_ERR_ARG;
  if (!in) return set_err(c, CRASH_ERR_ARG, "input is NULL");
  if (box < 0 || box >= c->n_boxes) return set_err(c, CRASH_ERR_ARG, "box index out of range");
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));
  const BoxMeta& m = c->meta[box];
  CK(cudaMemcpy(c->dep + 4 * m.cell_off, in, (size_t)m.ncell * 32, cudaMemcpyHostToDevice));
  return CRASH_OK;
}

// the chemistry's sub-step count of a separate per-cell update joins the totals
__global__ void k_add_substeps(const unsigned long long* budget, unsigned long long* totals, int n) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) totals[8 * b + 7] += budget[8 * b + 7];
}

extern "C" crash_status crash_chemistry(crash_ctx* c, double dt) {
  if (!c) return CRASH_ERR_ARG;
  if (!c->chem_pending)
    return set_err(c, CRASH_ERR_STATE, "crash_chemistry follows one step run with chemistry = 0");
  if (!(dt == c->last_dt)) return set_err(c, CRASH_ERR_ARG, "crash_chemistry needs the dt of its step");
  cudaSetDevice(c->device);
  StepArgs a = make_args(c, dt, 0);
  a.chemistry = 1;
  {
    NvtxRange chem_range("chemistry");
    launch_chemistry(a, c->stream);
  }
  k_add_substeps<<<(c->n_boxes + 127) / 128, 128, 0, c->stream>>>(c->budget, c->totals, c->n_boxes);
  CK(cudaGetLastError());
  c->launches += 2;
  c->chem_pending = false;
  return CRASH_OK;
}

// ---------------------------------------------------------------- timing
extern "C" crash_status crash_kernel_time(crash_ctx* c, double* ms, int64_t* launches) {
  if (!c || !ms || !launches) return set_err(c, CRASH_ERR_ARG, "NULL argument");
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));
  double acc = c->ms_accum;
  for (int i = 0; i < c->ev_used; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->events[i].first, c->events[i].second));
    acc += t;
  }
  c->ms_accum = acc;
  c->launches_accum += c->ev_used;
  c->ev_used = 0;
  *ms = c->ms_accum;
  *launches = c->launches_accum;
  return CRASH_OK;
}

extern "C" crash_status crash_reset_kernel_time(crash_ctx* c) {
  if (!c) return CRASH_ERR_ARG;
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));
  c->ev_used = 0;
  c->ms_accum = 0.0;
  c->launches_accum = 0;
  return CRASH_OK;
}

// ---------------------------------------------------------------- autotune
extern "C" crash_status crash_autotune(crash_ctx* c, double dt, const uint64_t* P, int* block,
                                       int* seg, int* resort, int* reg_cap, int* tile,
                                       int* sort_curve) {
  if (!c || !P) return CRASH_ERR_ARG;
  cudaSetDevice(c->device);
  // save the state and the step index so that trials leave no trace
  const size_t n = (size_t)c->n_cells;
  double* save = nullptr;
  CK(cudaMalloc(&save, n * 8 * 4));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(save, c->xHII, n * 8, cudaMemcpyDeviceToDevice));
  CK(cudaMemcpy(save + n, c->xHeII, n * 8, cudaMemcpyDeviceToDevice));
  CK(cudaMemcpy(save + 2 * n, c->xHeIII, n * 8, cudaMemcpyDeviceToDevice));
  CK(cudaMemcpy(save + 3 * n, c->T, n * 8, cudaMemcpyDeviceToDevice));
  // the diffuse field's counts too: trial steps re-emit and reset them
  double* save_rec = nullptr;
  if (c->any_rec) {
    CK(cudaMalloc(&save_rec, n * 24));
    CK(cudaMemcpy(save_rec, c->rec, n * 24, cudaMemcpyDeviceToDevice));
  }
  unsigned long long step0 = 0;
  CK(cudaMemcpy(&step0, c->step_dev, 8, cudaMemcpyDeviceToHost));
  crash_run_opts base = c->opts;
  crash_run_opts best = base;
  double best_ms = 1e300;
  // trials trace a window of about 2^26 packets (a quarter of a wavefront chunk) or less
  uint32_t win = 0xFFFFFFFFu;
  {
    int64_t tot = 0;
    for (int b = 0; b < c->n_boxes; ++b) tot += (int64_t)P[b];
    if (tot > ((int64_t)1 << 26)) {
      uint64_t mx = 1;
      for (int b = 0; b < c->n_boxes; ++b) mx = std::max<uint64_t>(mx, P[b] / (uint64_t)c->meta[b].n_src);
      win = (uint32_t)std::max<uint64_t>(1, (uint64_t)((double)mx * (double)((int64_t)1 << 26) / (double)tot));
    }
  }
  std::vector<int> blocks = {64, 128, 256};
  std::vector<int> segs = {0};
  std::vector<int> resorts = {0};
  std::vector<int> caps = {0};
  if (c->precision == CRASH_MIXED) {
    blocks = {128, 256};
    segs = {16, 32, 64};
    resorts = {1, 2};
    caps = {0, 1};
  }
  crash_status st = CRASH_OK;
  struct Trial { int bs, sg, rs, cap, tile; };
  std::vector<Trial> trials;
  for (int cap : caps)
    for (int bs : blocks)
      for (int sg : segs)
        for (int rs : resorts) trials.push_back({bs, sg, rs, cap, 0});
  if (c->precision == CRASH_MIXED) trials.push_back({256, 0, 1, 0, 1});
  // the grid of trials runs one launch per pass; the fastest configuration is
  // then tried once more with Hilbert-ordered bucket keys, and the fastest of
  // those once more as one persistent launch per step
  const int n_grid = (int)trials.size();
  for (int ti = 0; ti < n_grid + 2; ++ti) {
    const bool curve_trial = ti == n_grid, pers_trial = ti == n_grid + 1;
    if ((curve_trial || pers_trial) && (c->precision != CRASH_MIXED || best.tile || best_ms >= 1e300)) break;
    const Trial tr = ti >= n_grid ? Trial{best.block_size, best.seg_per_iter, best.resort_interval,
                                          best.reg_cap, best.tile}
                                  : trials[ti];
    crash_run_opts o = base;
    o.sort_curve = curve_trial ? 1 : (pers_trial ? best.sort_curve : 0);
    o.persistent = pers_trial ? 1 : 0;
    o.block_size = tr.bs;
    o.seg_per_iter = tr.sg;
    o.resort_interval = tr.rs;
    o.reg_cap = tr.cap;
    o.tile = tr.tile;
    o.pkt_begin = 0;
    o.pkt_end = win;
    o.chemistry = 0;
    o.use_graph = 0;
    o.timing = 0;
    c->opts = o;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    st = crash_step_batch(c, dt, P);                 // warm-up
    if (st == CRASH_OK) {
      cudaEventRecord(e0, c->stream);
      st = crash_step_batch(c, dt, P);
      cudaEventRecord(e1, c->stream);
    }
    cudaStreamSynchronize(c->stream);
    float ms = 0.f;
    if (st == CRASH_OK) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CRASH_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = base;
      best.block_size = tr.bs;
      best.seg_per_iter = tr.sg;
      best.resort_interval = tr.rs;
      best.reg_cap = tr.cap;
      best.tile = tr.tile;
      best.sort_curve = o.sort_curve;
      best.persistent = o.persistent;
    }
  }
  c->opts = best;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  cudaMemcpy(c->xHII, save, n * 8, cudaMemcpyDeviceToDevice);
  cudaMemcpy(c->xHeII, save + n, n * 8, cudaMemcpyDeviceToDevice);
  cudaMemcpy(c->xHeIII, save + 2 * n, n * 8, cudaMemcpyDeviceToDevice);
  cudaMemcpy(c->T, save + 3 * n, n * 8, cudaMemcpyDeviceToDevice);
  cudaMemcpy(c->step_dev, &step0, 8, cudaMemcpyHostToDevice);
  cudaFree(save);
  if (save_rec) {
    cudaMemcpy(c->rec, save_rec, n * 24, cudaMemcpyDeviceToDevice);
    cudaFree(save_rec);
  }
  c->step_host = step0;
  if (st != CRASH_OK) return st;
  if (block) *block = best.block_size;
  if (seg) *seg = best.seg_per_iter;
  if (resort) *resort = best.resort_interval;
  if (reg_cap) *reg_cap = best.reg_cap;
  if (tile) *tile = best.tile;
  if (sort_curve) *sort_curve = best.sort_curve;
  return CRASH_OK;
}
