// k_fp64.cu -- per-step preparation kernels and the FP64 transport kernel.
// Built with -fmad=false: every product and sum is rounded on its own, which
// makes the FP64 form reproduce the FP64 step specification bit for bit.
//
//   k_prep     one thread per cell: absorber densities frozen for the step
//              (Sec. 2: tau of a cell sums H I, He I and He II) and zeroed
//              deposit counters.
//   k_budget   one thread per source: the source's photons this step in
//              integer quanta, split over frequency bins (coloured packets,
//              Sec. 2) and over its N_p/N_t packets (Sec. 3.2).
//   k_trace_fp64  one thread per packet: isotropic direction, content, and
//              the cell-by-cell walk with Eq. 1 attenuation and int64
//              deposition until the packet is empty or leaves the grid.
//   k_rec_max, k_rec_select, k_rec_fp64  diffuse recombination field
//              (Sec. 2): the largest count over threshold (for the step's
//              quantum), this step's re-emitting cells, and one FP64 packet
//              per such cell walked like a source packet.
#include <math.h>

#include <algorithm>

#include "crash_internal.cuh"
#include "k_device.cuh"

using namespace crash;

// ------------------------------------------------------------------ prep
__global__ void k_prep(StepArgs a, int mixed) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < a.n_cells_total; i += stride) {
    int b = box_of_cell(a.boxes, a.n_boxes, i);
    double he = a.boxes[b].he;
    double nH = (double)a.nH[i];
    double nHe = nH * he;
    double x = a.xHII[i], y2 = a.xHeII[i], y3 = a.xHeIII[i];
    double aHI = nH * (1.0 - x);
    double aHeI = nHe * ((1.0 - y2) - y3);
    double aHeII = nHe * y2;
    if (mixed) {
      reinterpret_cast<float4*>(a.abs32)[i] =
          make_float4((float)aHI, (float)aHeI, (float)aHeII, 0.0f);
    } else {
      double2* p = reinterpret_cast<double2*>(a.abs64) + 2 * i;
      p[0] = make_double2(aHI, aHeI);
      p[1] = make_double2(aHeII, 0.0);
    }
    ulonglong2* d = reinterpret_cast<ulonglong2*>(a.dep) + 2 * i;
    d[0] = make_ulonglong2(0ull, 0ull);
    d[1] = make_ulonglong2(0ull, 0ull);
  }
}

void launch_prep(const StepArgs& a, int precision, cudaStream_t s) {
  int64_t blocks = (a.n_cells_total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  k_prep<<<(unsigned)blocks, 256, 0, s>>>(a, precision == CRASH_MIXED);
}

// ------------------------------------------------------------------ budget
__device__ __forceinline__ int box_of_source(const BoxMeta* b, int n, int s) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b[mid].src_off <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_budget(StepArgs a, int n_bins) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n_src_total) return;
  int b = box_of_source(a.boxes, a.n_boxes, s);
  const BoxMeta& M = a.boxes[b];
  // quantum q = 2^E with the step's photons of all the box's sources,
  // (sum of ndot) dt / q, at most 2^62
  double X = M.ndot_sum * a.dt;
  int E = X > 0.0 ? ceil_log2_dev(X) - 62 : 0;
  // the diffuse recombination field re-emits this step at most ncell times
  // the largest count over its threshold: the quantum also keeps that below
  // 2^62, and one more bit keeps sources plus re-emission below 2^62
  if (M.f_rec > 0.0) {
    const double rmax = __longlong_as_double((long long)a.rec_rmax[b]);
    if (rmax > 0.0) {
      const int Er = ceil_log2_dev(rmax * (double)M.ncell) - 62;
      E = Er > E ? Er : E;
    }
    E += 1;
  }
  long long B = llrint(ldexp(a.src_ndot[s] * a.dt, -E));
  long long Ns = (long long)M.pkts_per_src;
  double F = 0.0;
  long long prev = 0;
  for (int j = 0; j < n_bins; ++j) {
    long long Cj;
    if (j == n_bins - 1) {
      Cj = B;
    } else {
      F = F + a.src_frac[(int64_t)s * n_bins + j];
      Cj = (long long)floor((double)B * F);
      Cj = Cj > B ? B : Cj;
      Cj = Cj < prev ? prev : Cj;
    }
    long long Bj = Cj - prev;
    prev = Cj;
    a.src_base[(int64_t)s * n_bins + j] = Bj / Ns;
    a.src_rem[(int64_t)s * n_bins + j] = Bj % Ns;
  }
  if (s == M.src_off) {
    a.box_E[b] = E;
    a.budget[b * 8 + 5] = (unsigned long long)(long long)E;
    a.budget[b * 8 + 6] = (unsigned long long)(long long)M.heatF;
  }
}

void launch_budget(const StepArgs& a, const BinTables& t, cudaStream_t s) {
  int blocks = (a.n_src_total + 127) / 128;
  k_budget<<<blocks, 128, 0, s>>>(a, t.n_bins);
}

// ------------------------------------------------------------------ trace
struct Tally {
  unsigned long long emitted, absorbed, escaped, crossings, packets;
};

// per-box budget accumulation: warp-wide sums when the warp's packets share a
// box, per-lane atomics otherwise
__device__ __forceinline__ void flush_tally(const StepArgs& a, int b, Tally t) {
  unsigned mask = 0xFFFFFFFFu;
  int b0 = __shfl_sync(mask, b, 0);
  bool uniform = __all_sync(mask, b == b0 || b < 0);
  if (uniform) {
    t.emitted = warp_sum_u64(t.emitted);
    t.absorbed = warp_sum_u64(t.absorbed);
    t.escaped = warp_sum_u64(t.escaped);
    t.crossings = warp_sum_u64(t.crossings);
    t.packets = warp_sum_u64(t.packets);
    if ((threadIdx.x & 31) == 0 && b0 >= 0) {
      unsigned long long* g = a.budget + b0 * 8;
      if (t.emitted) atomicAdd(g + 0, t.emitted);
      if (t.absorbed) atomicAdd(g + 1, t.absorbed);
      if (t.escaped) atomicAdd(g + 2, t.escaped);
      if (t.crossings) atomicAdd(g + 3, t.crossings);
      if (t.packets) atomicAdd(g + 4, t.packets);
    }
  } else if (b >= 0) {
    unsigned long long* g = a.budget + b * 8;
    atomicAdd(g + 0, t.emitted);
    atomicAdd(g + 1, t.absorbed);
    atomicAdd(g + 2, t.escaped);
    atomicAdd(g + 3, t.crossings);
    atomicAdd(g + 4, t.packets);
  }
}

// Walk one packet from (px, py, pz) (grid units, inside or outside the box)
// along (dx, dy, dz) through the frozen FP64 absorbers (Amanatides & Woo
// 1987, ties x before y before z): per crossed cell with path l > 0, per bin
// Eq. 1 in integer quanta N' = rint(N e^-tau), the absorbed A = N - N' split
// by optical-depth share (Sec. 2), excess energy rounded once per cell.
// In a periodic box (Sec. 2) the walk re-enters through the opposite face and
// ends after the light-travel distance c dt (the last segment cut there),
// what the packet still holds then being counted as escaped.
// Deposits go to the grid, counts to tl; the content N is consumed.
template <int NBT, bool HE, bool HEAT>
__device__ __forceinline__ void walk_fp64(const StepArgs& a, const BinTables& t, const BoxMeta* M,
                                          int nb, double px, double py, double pz, double dx,
                                          double dy, double dz, long long* N, Tally& tl) {
  const int nx = M->nx, ny = M->ny, nz = M->nz;
  const double dl = M->dl;
  const int64_t coff = M->cell_off;
  int ix = (int)floor(px), iy = (int)floor(py), iz = (int)floor(pz);
  int sx, sy, sz;
  double tMx, tMy, tMz, tDx, tDy, tDz;
  if (dx > 0) { sx = 1; tMx = ((double)(ix + 1) - px) / dx; tDx = 1.0 / dx; }
  else if (dx < 0) { sx = -1; tMx = ((double)ix - px) / dx; tDx = -1.0 / dx; }
  else { sx = 0; tMx = INFINITY; tDx = INFINITY; }
  if (dy > 0) { sy = 1; tMy = ((double)(iy + 1) - py) / dy; tDy = 1.0 / dy; }
  else if (dy < 0) { sy = -1; tMy = ((double)iy - py) / dy; tDy = -1.0 / dy; }
  else { sy = 0; tMy = INFINITY; tDy = INFINITY; }
  if (dz > 0) { sz = 1; tMz = ((double)(iz + 1) - pz) / dz; tDz = 1.0 / dz; }
  else if (dz < 0) { sz = -1; tMz = ((double)iz - pz) / dz; tDz = -1.0 / dz; }
  else { sz = 0; tMz = INFINITY; tDz = INFINITY; }
  bool escaped = (ix < 0 || ix >= nx || iy < 0 || iy >= ny || iz < 0 || iz >= nz);
  bool done = escaped;
  double tcur = 0.0;
  // a path of length L crosses at most (|dx| + |dy| + |dz|) L + 3 < 2 L + 3 faces
  const bool per = M->periodic != 0;
  const double tlim = per ? (CRASH_C_LIGHT * a.dt) / dl : INFINITY;
  const int64_t max_iter = per ? (int64_t)(2.0 * tlim) + 4 : (int64_t)(nx + ny + nz + 3);
  int64_t it = 0;
  for (; !done && it < max_iter; ++it) {
    int ax = 0;
    double tn = tMx;
    if (tMy < tn) { ax = 1; tn = tMy; }
    if (tMz < tn) { ax = 2; tn = tMz; }
    const bool stop = tn >= tlim;
    if (stop) tn = tlim;
    const double seg = tn - tcur;
    if (seg > 0) {
      const int64_t cell = coff + (int64_t)ix + (int64_t)nx * ((int64_t)iy + (int64_t)ny * iz);
      const double l = seg * dl;
      const double2 a01 = __ldg(reinterpret_cast<const double2*>(a.abs64) + 2 * cell);
      const double nHI = a01.x;
      double nHeI = 0.0, nHeII = 0.0;
      if (HE) {
        nHeI = a01.y;
        nHeII = __ldg(reinterpret_cast<const double2*>(a.abs64) + 2 * cell + 1).x;
      }
      long long dHI = 0, dHeI = 0, dHeII = 0, left = 0;
      double heat = 0.0;
#pragma unroll
      for (int j = 0; j < (NBT > 0 ? NBT : CRASH_MAX_BINS); ++j) {
        if (NBT == 0 && j >= nb) break;
        const double kHI = nHI * t.sigma[0][j];
        double kap = kHI, kHeI = 0.0, kHeII = 0.0;
        if (HE) {
          kHeI = nHeI * t.sigma[1][j];
          kHeII = nHeII * t.sigma[2][j];
          kap = (kHI + kHeI) + kHeII;
        }
        const double f = exp_neg_spec(l * kap);
        const long long Nj = N[j];
        long long Np = llrint((double)Nj * f);
        Np = Np > Nj ? Nj : Np;
        const long long A = Nj - Np;
        N[j] = Np;
        left |= Np;
        if (A > 0) {
          long long A1 = 0, A2 = 0;
          if (HE) {
            A1 = llrint((double)A * (kHeI / kap));
            A1 = A1 > A ? A : A1;
            A2 = llrint((double)A * (kHeII / kap));
            A2 = A2 > A - A1 ? A - A1 : A2;
          }
          const long long A0 = A - A1 - A2;
          dHI += A0;
          dHeI += A1;
          dHeII += A2;
          if (HEAT) {
            if (HE)
              heat += ((double)A0 * t.wheat[0][j] + (double)A1 * t.wheat[1][j]) +
                      (double)A2 * t.wheat[2][j];
            else
              heat += (double)A0 * t.wheat[0][j];
          }
        }
      }
      unsigned long long* dp = a.dep + 4 * cell;
      if (dHI) atomicAdd(dp + 0, (unsigned long long)dHI);
      if (HE) {
        if (dHeI) atomicAdd(dp + 1, (unsigned long long)dHeI);
        if (dHeII) atomicAdd(dp + 2, (unsigned long long)dHeII);
      }
      if (HEAT && !M->isothermal) {
        long long h = llrint(heat);
        if (h) atomicAdd(dp + 3, (unsigned long long)h);
      }
      tl.absorbed += (unsigned long long)(dHI + dHeI + dHeII);
      tl.crossings += 1;
      if (left == 0) { done = true; break; }
    }
    if (stop) { escaped = true; done = true; break; }
    tcur = tn;
    if (ax == 0) { tMx += tDx; ix += sx; }
    else if (ax == 1) { tMy += tDy; iy += sy; }
    else { tMz += tDz; iz += sz; }
    if (per) {
      ix = ix < 0 ? nx - 1 : (ix >= nx ? 0 : ix);
      iy = iy < 0 ? ny - 1 : (iy >= ny ? 0 : iy);
      iz = iz < 0 ? nz - 1 : (iz >= nz ? 0 : iz);
    } else {
      escaped = (ix < 0 || ix >= nx || iy < 0 || iy >= ny || iz < 0 || iz >= nz);
    }
    if (escaped) done = true;
  }
  if (escaped) {
    for (int j = 0; j < nb; ++j) tl.escaped += (unsigned long long)N[j];
  } else if (!done) {
    atomicOr(a.err, ERR_DDA_LIMIT);
  }
}

template <int NBT, bool HE, bool HEAT>
__global__ void __launch_bounds__(256) k_trace_fp64(StepArgs a, BinTables t) {
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  Tally tl{0, 0, 0, 0, 0};
  int b = -1;
  if (gid < a.total_packets) {
    b = box_of_packet(a.boxes, a.n_boxes, gid);
    const BoxMeta* M = a.boxes + b;
    const int64_t local = gid - M->pkt_off;
    const uint32_t W = M->win_hi - M->win_lo;
    const int s_local = (int)(local / W);
    const uint32_t p = M->win_lo + (uint32_t)(local - (int64_t)s_local * W);
    const int s = M->src_off + s_local;
    double dx, dy, dz;
    const uint32_t step = (uint32_t)*a.step_dev;
    if (!iso_direction(M->seed, step, (uint32_t)s_local, p, dx, dy, dz)) {
      atomicOr(a.err, ERR_DIRECTION);
    } else {
      long long N[NBT > 0 ? NBT : CRASH_MAX_BINS];
      for (int j = 0; j < nb; ++j) {
        long long base = a.src_base[(int64_t)s * nb + j];
        long long rem = a.src_rem[(int64_t)s * nb + j];
        N[j] = base + ((long long)p < rem ? 1 : 0);
        tl.emitted += (unsigned long long)N[j];
      }
      tl.packets = 1;
      walk_fp64<NBT, HE, HEAT>(a, t, M, nb, a.src_pos[3 * s], a.src_pos[3 * s + 1],
                               a.src_pos[3 * s + 2], dx, dy, dz, N, tl);
    }
  }
  flush_tally(a, b, tl);
}

// One re-emission packet per entry of this step's list (diffuse
// recombination field): start point and direction from the cell's Philox
// counters, the photons of each species in its bin, then the same walk as a
// source packet.  Entries are read in any order: the integer deposits and
// counts do not depend on it.
template <int NBT, bool HE, bool HEAT>
__global__ void __launch_bounds__(256) k_rec_fp64(StepArgs a, BinTables t) {
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const int64_t n = (int64_t)*a.rec_count;
  const uint32_t step = (uint32_t)*a.step_dev;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = base + threadIdx.x;
    Tally tl{0, 0, 0, 0, 0};
    int b = -1;
    if (e < n) {
      const long long* L = a.rec_list + 4 * e;
      const int64_t g = L[0];
      b = box_of_cell(a.boxes, a.n_boxes, g);
      const BoxMeta* M = a.boxes + b;
      const int64_t cell = g - M->cell_off;
      double ox, oy, oz, dx, dy, dz;
      rec_offsets(M->seed, step, cell, ox, oy, oz);
      if (!iso_direction(M->seed, step, rec_src_id(cell), (uint32_t)cell, dx, dy, dz)) {
        atomicOr(a.err, ERR_DIRECTION);
      } else {
        long long N[NBT > 0 ? NBT : CRASH_MAX_BINS];
        for (int j = 0; j < nb; ++j) N[j] = 0;
        for (int s = 0; s < 3; ++s)
          if (a.rec_bin[s] >= 0) N[a.rec_bin[s]] += L[1 + s];
        for (int j = 0; j < nb; ++j) tl.emitted += (unsigned long long)N[j];
        tl.packets = 1;
        const int64_t ix = cell % M->nx, iy = (cell / M->nx) % M->ny, iz = cell / ((int64_t)M->nx * M->ny);
        walk_fp64<NBT, HE, HEAT>(a, t, M, nb, (double)ix + ox, (double)iy + oy, (double)iz + oz,
                                 dx, dy, dz, N, tl);
      }
    }
    flush_tally(a, b, tl);
  }
}

// The largest count over its threshold in each box (for the step's
// quantum).  Counts are >= 0 doubles, whose bit patterns order like the
// values, so an integer atomicMax gives the same result in any order.
__device__ __forceinline__ bool rec_over(const StepArgs& a, const BoxMeta* M, int64_t g, int s,
                                         double& v) {
  const double V = (M->dl * M->dl) * M->dl;
  const double nH = (double)a.nH[g];
  const double atoms = s == 0 ? nH * V : nH * M->he * V;
  v = a.rec[(int64_t)s * a.n_cells_total + g];
  return atoms > 0 && v > 0 && v >= M->f_rec * atoms;
}

__global__ void k_rec_max(StepArgs a) {
  const int64_t n = a.n_cells_total;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int b = box_of_cell(a.boxes, a.n_boxes, g);
    const BoxMeta* M = a.boxes + b;
    if (!(M->f_rec > 0.0)) continue;
    double m = 0.0;
    for (int s = 0; s < 3; ++s) {
      double v;
      if (rec_over(a, M, g, s, v) && v > m) m = v;
    }
    if (m > 0.0) atomicMax(a.rec_rmax + b, (unsigned long long)__double_as_longlong(m));
  }
}

void launch_rec_max(const StepArgs& a, cudaStream_t s) {
  cudaMemsetAsync(a.rec_rmax, 0, sizeof(unsigned long long) * a.n_boxes, s);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((a.n_cells_total + 255) / 256, (int64_t)sms * 8);
  k_rec_max<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a);
}

// This step's re-emitting cells: where the recombinations to the ground
// state of a species reached f_rec times the element's atoms in the cell,
// its photons (in the step's quanta) leave as one packet and its count
// restarts from 0.  Species without a bin at or above their threshold are
// not emitted (their count restarts all the same).  One list entry per cell
// that emits anything.
__global__ void k_rec_select(StepArgs a) {
  const int64_t n = a.n_cells_total;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int b = box_of_cell(a.boxes, a.n_boxes, g);
    const BoxMeta* M = a.boxes + b;
    if (!(M->f_rec > 0.0)) continue;
    const double q = ldexp(1.0, a.box_E[b]);
    long long Nq[3] = {0, 0, 0};
    bool any = false;
    for (int s = 0; s < 3; ++s) {
      double v;
      if (rec_over(a, M, g, s, v)) {
        Nq[s] = a.rec_bin[s] >= 0 ? llrint(v / q) : 0;
        a.rec[(int64_t)s * n + g] = 0.0;
        any = true;
      }
    }
    if (!any || (Nq[0] | Nq[1] | Nq[2]) == 0) continue;
    const unsigned slot = atomicAdd(a.rec_count, 1u);
    long long* L = a.rec_list + 4 * (int64_t)slot;
    L[0] = g;
    L[1] = Nq[0];
    L[2] = Nq[1];
    L[3] = Nq[2];
  }
}

void launch_rec_select(const StepArgs& a, cudaStream_t s) {
  cudaMemsetAsync(a.rec_count, 0, sizeof(unsigned), s);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((a.n_cells_total + 255) / 256, (int64_t)sms * 8);
  k_rec_select<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a);
}

template <int NBT, bool HE, bool HEAT>
static void launch_r(const StepArgs& a, const BinTables& t, cudaStream_t s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_rec_fp64<NBT, HE, HEAT><<<(unsigned)(sms * 4), 256, 0, s>>>(a, t);
}

void launch_rec_fp64(const StepArgs& a, const BinTables& t, cudaStream_t s) {
  const bool he = a.any_he != 0, heat = a.any_heat != 0;
  if (t.n_bins == 1) {
    if (he) { if (heat) launch_r<1, true, true>(a, t, s); else launch_r<1, true, false>(a, t, s); }
    else { if (heat) launch_r<1, false, true>(a, t, s); else launch_r<1, false, false>(a, t, s); }
  } else if (t.n_bins == 8) {
    if (he) { if (heat) launch_r<8, true, true>(a, t, s); else launch_r<8, true, false>(a, t, s); }
    else { if (heat) launch_r<8, false, true>(a, t, s); else launch_r<8, false, false>(a, t, s); }
  } else {
    if (he) { if (heat) launch_r<0, true, true>(a, t, s); else launch_r<0, true, false>(a, t, s); }
    else { if (heat) launch_r<0, false, true>(a, t, s); else launch_r<0, false, false>(a, t, s); }
  }
}

template <int NBT, bool HE, bool HEAT>
static void launch_t(const StepArgs& a, const BinTables& t, int block, cudaStream_t s) {
  int64_t blocks = (a.total_packets + block - 1) / block;
  k_trace_fp64<NBT, HE, HEAT><<<(unsigned)blocks, block, 0, s>>>(a, t);
}

void launch_trace_fp64(const StepArgs& a, const BinTables& t, int block, cudaStream_t s) {
  if (a.total_packets <= 0) return;
  if (block <= 0) block = 128;
  // the H+He kernels are exact for pure-H boxes too (their He terms are
  // +0), and isothermal boxes skip the heating deposit at run time
  const bool he = a.any_he != 0, heat = a.any_heat != 0;
  if (t.n_bins == 1) {
    if (he) { if (heat) launch_t<1, true, true>(a, t, block, s); else launch_t<1, true, false>(a, t, block, s); }
    else { if (heat) launch_t<1, false, true>(a, t, block, s); else launch_t<1, false, false>(a, t, block, s); }
  } else if (t.n_bins == 8) {
    if (he) { if (heat) launch_t<8, true, true>(a, t, block, s); else launch_t<8, true, false>(a, t, block, s); }
    else { if (heat) launch_t<8, false, true>(a, t, block, s); else launch_t<8, false, false>(a, t, block, s); }
  } else {
    if (he) { if (heat) launch_t<0, true, true>(a, t, block, s); else launch_t<0, true, false>(a, t, block, s); }
    else { if (heat) launch_t<0, false, true>(a, t, block, s); else launch_t<0, false, false>(a, t, block, s); }
  }
}
