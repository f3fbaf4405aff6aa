// k_noalloc.cu -- transport of one grid for one step that allocates no
// device memory: for callers that cannot call cudaMalloc (code running
// inside another framework's memory pool or under a strict memory budget,
// plug-ins that may only use buffers handed to them, processes that must not
// grow their footprint after start-up).  The caller passes the absorbers and
// the deposit buffer; every scratch buffer of the step (the wavefront packet
// queue, the per-source budget tables, the counters) lives in the file-scope
// array below, which every GPU that loads the library holds until the
// process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "crash_internal.cuh"

namespace {

// capacity of the static scratch
constexpr int64_t kQueuePackets = 1 << 16;         // packets held by each queue buffer
constexpr int kMaxSources = CRASH_NOALLOC_MAX_SOURCES;
constexpr int64_t kRecordBytes = 32 + 8 * CRASH_MAX_BINS;   // largest record (16 bins)

constexpr int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }
constexpr int64_t kOffRec0 = 0;
constexpr int64_t kOffRec1 = kOffRec0 + align256(kQueuePackets * kRecordBytes);
constexpr int64_t kOffCount = kOffRec1 + align256(kQueuePackets * kRecordBytes);
constexpr int64_t kOffErr = kOffCount + 256;
constexpr int64_t kOffStep = kOffErr + 256;
constexpr int64_t kOffMeta = kOffStep + 256;
constexpr int64_t kOffBoxE = kOffMeta + align256(sizeof(BoxMeta));
constexpr int64_t kOffBudget = kOffBoxE + 256;
constexpr int64_t kOffNdot = kOffBudget + 256;
constexpr int64_t kOffFrac = kOffNdot + align256(8 * kMaxSources);
constexpr int64_t kOffBase = kOffFrac + align256(8 * (int64_t)kMaxSources * CRASH_MAX_BINS);
constexpr int64_t kOffRem = kOffBase + align256(8 * (int64_t)kMaxSources * CRASH_MAX_BINS);
constexpr int64_t kOffPos32 = kOffRem + align256(8 * (int64_t)kMaxSources * CRASH_MAX_BINS);
constexpr int64_t kOffCell = kOffPos32 + align256(4 * 3 * kMaxSources);
constexpr int64_t kScratchBytes = kOffCell + align256(4 * 3 * kMaxSources);

// the scratch: ~21 MB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of g_noalloc_scratch per device, looked up on first use
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

thread_local std::string g_noalloc_error;

crash_status fail(crash_status st, const std::string& m) {
  g_noalloc_error = m;
  return st;
}

}  // namespace

extern "C" const char* crash_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" crash_status crash_transport_noalloc(const crash_grid_desc* grid, int n_src,
                                                const double* pos_cells, const double* ndot,
                                                int n_bins, const double* bin_eV,
                                                const double* bin_frac, double dt_s,
                                                uint64_t step_index, uint64_t packets_per_step,
                                                int seg_per_pass, const float* absorbers_dev,
                                                unsigned long long* deposits_dev,
                                                int64_t* budget_out, void* stream) {
  // ---- host-side argument checks (nothing reaches the GPU before these pass)
  if (!grid || !pos_cells || !ndot || !bin_eV || !bin_frac || !absorbers_dev || !deposits_dev ||
      !budget_out)
    return fail(CRASH_ERR_ARG, "NULL argument");
  // the transport gathers absorbers as float4 and adds deposits with 64-bit
  // reductions: a misaligned buffer (an offset view, say) would fault on the
  // GPU, so it is refused here, before anything is launched
  if (((uintptr_t)absorbers_dev & 15u) != 0)
    return fail(CRASH_ERR_ARG, "absorbers_dev must be 16-byte aligned");
  if (((uintptr_t)deposits_dev & 7u) != 0)
    return fail(CRASH_ERR_ARG, "deposits_dev must be 8-byte aligned");
  const crash_grid_desc& d = *grid;
  if (d.nx < 1 || d.ny < 1 || d.nz < 1 || !(d.box_cm > 0))
    return fail(CRASH_ERR_ARG, "grid dimensions and box_cm must be positive");
  if (d.f_rec != 0.0)
    return fail(CRASH_ERR_ARG, "the allocation-free call traces source packets only: f_rec must be 0");
  if (d.nx > 65535 || d.ny > 65535 || d.nz > 65535 || (int64_t)d.nx * d.ny * d.nz >= ((int64_t)1 << 31))
    return fail(CRASH_ERR_OVERFLOW, "each axis <= 65535 cells and < 2^31 cells");
  if (n_src < 1 || n_src > kMaxSources)
    return fail(CRASH_ERR_OVERFLOW, "n_src must be in [1, CRASH_NOALLOC_MAX_SOURCES = " +
                                        std::to_string(kMaxSources) + "]");
  if (n_bins < 1 || n_bins > CRASH_MAX_BINS) return fail(CRASH_ERR_OVERFLOW, "n_bins must be in [1, 16]");
  if (!(dt_s > 0) || !isfinite(dt_s)) return fail(CRASH_ERR_ARG, "dt must be positive");
  if (packets_per_step == 0 || packets_per_step % (uint64_t)n_src)
    return fail(CRASH_ERR_ARG, "packets_per_step must be a positive multiple of n_src");
  if (packets_per_step > (uint64_t)CRASH_NOALLOC_MAX_PACKETS)
    return fail(CRASH_ERR_OVERFLOW, "packets_per_step above CRASH_NOALLOC_MAX_PACKETS (2^30): split the "
                                    "step into calls over packet windows of a context instead");
  const uint64_t Ns = packets_per_step / (uint64_t)n_src;
  if (seg_per_pass < 0) return fail(CRASH_ERR_ARG, "seg_per_pass must be >= 0");
  for (int s = 0; s < n_src; ++s) {
    const double* p = pos_cells + 3 * s;
    if (!(p[0] >= 0 && p[0] < d.nx && p[1] >= 0 && p[1] < d.ny && p[2] >= 0 && p[2] < d.nz))
      return fail(CRASH_ERR_ARG, "source position outside the grid");
    if (!(ndot[s] >= 0) || !isfinite(ndot[s])) return fail(CRASH_ERR_ARG, "source rates must be finite and >= 0");
    for (int j = 0; j < n_bins; ++j)
      if (!(bin_frac[(size_t)s * n_bins + j] >= 0)) return fail(CRASH_ERR_ARG, "bin fractions must be >= 0");
  }
  for (int j = 0; j < n_bins; ++j)
    if (!(bin_eV[j] > 0)) return fail(CRASH_ERR_ARG, "bin energies must be positive");

  // ---- device address of the scratch (once per device, that device current)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(CRASH_ERR_CUDA, "no usable current CUDA device");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return fail(CRASH_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = (unsigned char*)ptr;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;

  // ---- tables and per-step constants (host), copied into the scratch
  BinTables t;
  memset(&t, 0, sizeof t);
  int heatF = 0;
  cross_sections(n_bins, bin_eV, t, heatF);
  BoxMeta m;
  memset(&m, 0, sizeof m);
  m.nx = d.nx; m.ny = d.ny; m.nz = d.nz;
  m.isothermal = d.isothermal ? 1 : 0;
  m.cell_off = 0;
  m.ncell = (int64_t)d.nx * d.ny * d.nz;
  m.dl = d.box_cm / d.nx;
  m.dlf = (float)m.dl;
  m.he = d.he_over_h;
  m.seed = d.seed;
  m.caseB = d.caseB ? 1 : 0;
  m.src_off = 0;
  m.n_src = n_src;
  m.heatF = heatF;
  double sum = 0.0;
  for (int s = 0; s < n_src; ++s) sum += ndot[s];
  m.ndot_sum = sum;
  m.pkts_per_src = Ns;
  m.win_lo = 0;
  m.win_hi = (uint32_t)Ns;
  m.pkt_off = 0;
  m.pkt_count = (int64_t)packets_per_step;
  m.max_iter = d.nx + d.ny + d.nz + 3;
  std::vector<float> pos32(3 * (size_t)n_src);
  std::vector<int> cell(3 * (size_t)n_src);
  for (int i = 0; i < 3 * n_src; ++i) {
    pos32[i] = (float)pos_cells[i];
    cell[i] = (int)floor(pos_cells[i]);
  }
  const unsigned long long step64 = step_index;
  const int zero = 0;
  struct Copy { int64_t off; const void* src; size_t bytes; };
  const Copy copies[] = {
      {kOffMeta, &m, sizeof m},
      {kOffStep, &step64, 8},
      {kOffErr, &zero, sizeof zero},
      {kOffNdot, ndot, 8 * (size_t)n_src},
      {kOffFrac, bin_frac, 8 * (size_t)n_src * n_bins},
      {kOffPos32, pos32.data(), 4 * pos32.size()},
      {kOffCell, cell.data(), 4 * cell.size()},
  };
  // host buffers are pageable: each copy is staged before the call returns
  for (const Copy& c : copies) {
    cudaError_t e = cudaMemcpyAsync(base + c.off, c.src, c.bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(CRASH_ERR_CUDA, std::string("copy into scratch: ") + cudaGetErrorString(e));
  }
  // the budget of this call starts at zero; the queue counters are cleared
  // by the wavefront launcher for every chunk
  {
    const cudaError_t e = cudaMemsetAsync(base + kOffBudget, 0, 64, s);
    if (e != cudaSuccess) return fail(CRASH_ERR_CUDA, std::string("clearing the budget: ") + cudaGetErrorString(e));
  }

  StepArgs a;
  memset(&a, 0, sizeof a);
  a.boxes = (const BoxMeta*)(base + kOffMeta);
  a.n_boxes = 1;
  a.step_dev = (unsigned long long*)(base + kOffStep);
  a.dt = dt_s;
  a.total_packets = (int64_t)packets_per_step;
  a.src_ndot = (const double*)(base + kOffNdot);
  a.src_frac = (const double*)(base + kOffFrac);
  a.src_base = (int64_t*)(base + kOffBase);
  a.src_rem = (int64_t*)(base + kOffRem);
  a.src_pos32 = (const float*)(base + kOffPos32);
  a.src_cell = (const int*)(base + kOffCell);
  a.box_E = (int*)(base + kOffBoxE);
  a.n_src_total = n_src;
  a.abs32 = const_cast<float*>(absorbers_dev);
  a.dep = deposits_dev;
  a.n_cells_total = m.ncell;
  a.budget = (unsigned long long*)(base + kOffBudget);
  a.err = (int*)(base + kOffErr);
  a.any_he = d.he_over_h > 0;
  a.any_heat = !d.isothermal;
  crash_run_opts o;
  crash_default_opts(&o);
  o.seg_per_iter = seg_per_pass;
  o.wavefront = 1;
  o.chemistry = 0;

  launch_budget(a, t, s);
  const int nk = launch_trace_mixed_external(a, t, o, (char*)(base + kOffRec0), (char*)(base + kOffRec1),
                                             (unsigned*)(base + kOffCount), kQueuePackets, m.max_iter, s);
  if (nk < 0) return fail(CRASH_ERR_CUDA, "transport launch failed");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CRASH_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));

  // ---- wait, then report the budget and any device-side limit
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(CRASH_ERR_CUDA, std::string("transport: ") + cudaGetErrorString(e));
  unsigned long long bud[8];
  int err = 0;
  e = cudaMemcpy(bud, base + kOffBudget, sizeof bud, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&err, base + kOffErr, sizeof err, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(CRASH_ERR_CUDA, std::string("read back: ") + cudaGetErrorString(e));
  for (int i = 0; i < 8; ++i) budget_out[i] = (int64_t)bud[i];
  if (err) return fail(CRASH_ERR_TIMEOUT, "device-side limit hit (DDA bound, direction draws or queue)");
  return CRASH_OK;
}
