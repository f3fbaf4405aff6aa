// k_mixed.cu -- mixed-precision transport: FP32 traversal, segment lengths
// and attenuation, exact int64 photon bookkeeping, FP64 only for the
// direction draw (so that every packet flies along the same direction as in
// the FP64 form).
//
// Per crossed cell and bin j (Sec. 2, Eq. 1): tau_j = l sum_s n_s sigma_s,j;
// the absorbed count A_j = rint(N_j (1 - e^-tau_j)) is formed in integer
// arithmetic from a 0.32 fixed-point absorption fraction, so N' = N - A
// keeps the photon budget exact; the species split (Sec. 2) and the
// heating energy are accumulated in FP32 over the bins and rounded once per
// cell, H I taking the remainder.
//
// Two launch shapes:
//   * one thread per packet (opts.wavefront = 0): emit and trace to the end;
//   * wavefront (default): the emission kernel traces every packet for at
//     most S DDA steps and appends the survivors to a device queue; pass
//     kernels (persistent, grid-stride over the live count held in device
//     memory) advance the queue S steps at a time until it is empty.  Every
//     R passes the queue is re-sorted by Morton order of its 8^3-cell bucket
//     and direction octant (one-pass counting sort), so that the packets a
//     warp holds gather neighbouring cells.  Deposits are integer sums, so
//     the processing order never changes a result.
// The launch sequence depends only on the grid sizes and S, never on data,
// so a step is capturable in a CUDA graph.
#include <math.h>

#include "crash_internal.cuh"
#include "k_device.cuh"

using namespace crash;

namespace {

struct WF {
  int64_t cap = 0;
  int nb = 0;
  uint2* cb[2] = {nullptr, nullptr};     // (ix | iy << 16, iz | box << 16)
  float4* td[2] = {nullptr, nullptr};    // (tMx, tMy, tMz, dx): distances to the next faces
  float2* dyz[2] = {nullptr, nullptr};   // (dy, dz)
  long long* N[2] = {nullptr, nullptr};  // [bin][cap] packet contents
  unsigned* count = nullptr;             // [4]: live counts of buffers 0 and 1
  unsigned* key = nullptr;               // [cap] sort key per packet
  unsigned* rank = nullptr;              // [cap] rank inside its key
  unsigned* bcount = nullptr;            // [n_keys]
  unsigned* boff = nullptr;              // [n_keys]
  unsigned* bsum = nullptr;              // [1024]
  int64_t n_keys = 0;
};

struct WFArgs {
  uint2* cb_in; float4* td_in; float2* dyz_in; long long* N_in;
  uint2* cb_out; float4* td_out; float2* dyz_out; long long* N_out;
  const unsigned* count_in;
  unsigned* count_out;
  int64_t cap;
};

struct Tally {
  unsigned long long emitted, absorbed, escaped, crossings, packets;
};

__device__ __forceinline__ void flush_warp(const StepArgs& a, int b, Tally& t) {
  const unsigned full = 0xFFFFFFFFu;
  const int b0 = __shfl_sync(full, b, 0);
  if (__all_sync(full, b == b0 || b < 0)) {
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
    if (t.emitted) atomicAdd(g + 0, t.emitted);
    if (t.absorbed) atomicAdd(g + 1, t.absorbed);
    if (t.escaped) atomicAdd(g + 2, t.escaped);
    if (t.crossings) atomicAdd(g + 3, t.crossings);
    if (t.packets) atomicAdd(g + 4, t.packets);
  }
  t = Tally{0, 0, 0, 0, 0};
}

// round(N * G / 2^32) for a 0.32 fixed-point fraction G < 2^32 (result <= N)
__device__ __forceinline__ long long mul_frac(long long N, unsigned G) {
  const unsigned long long n = (unsigned long long)N;
  const unsigned long long lo = (n & 0xFFFFFFFFull) * (unsigned long long)G;
  const unsigned long long hi = (n >> 32) * (unsigned long long)G;
  return (long long)(hi + ((lo + 0x80000000ull) >> 32));
}

// 1 - exp(-tau) in FP32 with small relative error for small tau
__device__ __forceinline__ float absorbed_fraction(float tau) {
  if (tau < 0.05f) {
    return tau * (1.0f - 0.5f * tau * (1.0f - (1.0f / 3.0f) * tau * (1.0f - 0.25f * tau)));
  }
  return 1.0f - __expf(-tau);
}

enum { ALIVE = 0, ABSORBED = 1, ESCAPED = 2 };

// Advance one packet by at most max_iter DDA steps.  tM* are the distances
// (in cells, along the ray) from the current point to the next x/y/z face;
// they are re-based at every step so that FP32 keeps their precision.
template <int NBT, bool HE, bool HEAT>
__device__ __forceinline__ int trace_mixed(int& ix, int& iy, int& iz, float& tMx, float& tMy,
                                           float& tMz, const float dx, const float dy,
                                           const float dz, long long* N, const BoxMeta* M,
                                           const StepArgs& a, const BinTables& t, const int nb,
                                           const int max_iter, Tally& tl) {
  const int nx = M->nx, ny = M->ny, nz = M->nz;
  const float tDx = dx != 0.f ? 1.0f / fabsf(dx) : INFINITY;
  const float tDy = dy != 0.f ? 1.0f / fabsf(dy) : INFINITY;
  const float tDz = dz != 0.f ? 1.0f / fabsf(dz) : INFINITY;
  const int sx = dx > 0.f ? 1 : -1, sy = dy > 0.f ? 1 : -1, sz = dz > 0.f ? 1 : -1;
  const float dl = (float)M->dl;
  const int64_t coff = M->cell_off;
  const bool heat_box = HEAT && !M->isothermal;
  const float4* __restrict__ abs32 = reinterpret_cast<const float4*>(a.abs32);
  for (int it = 0; it < max_iter; ++it) {
    const float seg = fminf(tMx, fminf(tMy, tMz));
    const int ax = (tMx <= tMy && tMx <= tMz) ? 0 : (tMy <= tMz ? 1 : 2);
    if (seg > 0.f) {
      const int local = ix + nx * (iy + ny * iz);
      const int64_t cell = coff + local;
      const float4 ab = __ldg(abs32 + cell);
      const float l = seg * dl;
      const float tHI = l * ab.x, tHeI = l * ab.y, tHeII = l * ab.z;
      long long Atot = 0, left = 0;
      float fHeI = 0.f, fHeII = 0.f, fheat = 0.f;
#pragma unroll
      for (int j = 0; j < (NBT > 0 ? NBT : CRASH_MAX_BINS); ++j) {
        if (NBT == 0 && j >= nb) break;
        const float k0 = tHI * t.sigma32[0][j];
        float tau = k0, k1 = 0.f, k2 = 0.f;
        if (HE) {
          k1 = tHeI * t.sigma32[1][j];
          k2 = tHeII * t.sigma32[2][j];
          tau = (k0 + k1) + k2;
        }
        long long Nj = N[j];
        if (tau > 0.f && Nj > 0) {
          const float g = absorbed_fraction(tau);
          const long long A = g >= 1.0f ? Nj : mul_frac(Nj, (unsigned)(g * 4294967296.0f));
          Nj -= A;
          N[j] = Nj;
          Atot += A;
          if (HE || HEAT) {
            const float Af = (float)A;
            const float inv = __frcp_rn(tau);
            if (HE) {
              fHeI += Af * (k1 * inv);
              fHeII += Af * (k2 * inv);
            }
            if (HEAT) {
              if (HE)
                fheat += Af * ((k0 * t.wheat32[0][j] + k1 * t.wheat32[1][j] + k2 * t.wheat32[2][j]) * inv);
              else
                fheat += Af * t.wheat32[0][j];
            }
          }
        }
        left |= Nj;
      }
      if (Atot) {
        long long dHeI = 0, dHeII = 0;
        if (HE) {
          dHeI = __float2ll_rn(fHeI);
          dHeI = dHeI > Atot ? Atot : dHeI;
          dHeII = __float2ll_rn(fHeII);
          dHeII = dHeII > Atot - dHeI ? Atot - dHeI : dHeII;
        }
        const long long dHI = Atot - dHeI - dHeII;
        unsigned long long* dp = a.dep + 4 * cell;
        if (dHI) atomicAdd(dp + 0, (unsigned long long)dHI);
        if (dHeI) atomicAdd(dp + 1, (unsigned long long)dHeI);
        if (dHeII) atomicAdd(dp + 2, (unsigned long long)dHeII);
        if (heat_box) {
          const long long h = __float2ll_rn(fheat);
          if (h) atomicAdd(dp + 3, (unsigned long long)h);
        }
        tl.absorbed += (unsigned long long)Atot;
      }
      tl.crossings += 1;
      if (left == 0) return ABSORBED;
    }
    tMx -= seg;
    tMy -= seg;
    tMz -= seg;
    if (ax == 0) {
      tMx = tDx; ix += sx;
      if ((unsigned)ix >= (unsigned)nx) return ESCAPED;
    } else if (ax == 1) {
      tMy = tDy; iy += sy;
      if ((unsigned)iy >= (unsigned)ny) return ESCAPED;
    } else {
      tMz = tDz; iz += sz;
      if ((unsigned)iz >= (unsigned)nz) return ESCAPED;
    }
  }
  return ALIVE;
}

// warp-aggregated append of surviving packets to the output queue
__device__ __forceinline__ long long append_slot(bool alive, unsigned* count_out) {
  const unsigned full = 0xFFFFFFFFu;
  const unsigned m = __ballot_sync(full, alive);
  if (m == 0) return -1;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(count_out, (unsigned)__popc(m));
  base = __shfl_sync(full, base, leader);
  if (!alive) return -1;
  return (long long)base + __popc(m & ((1u << lane) - 1u));
}

template <int NBT>
__device__ __forceinline__ void store_packet(const WFArgs& w, long long slot, int ix, int iy, int iz,
                                             int box, float tMx, float tMy, float tMz, float dx,
                                             float dy, float dz, const long long* N, int nb) {
  w.cb_out[slot] = make_uint2((unsigned)ix | ((unsigned)iy << 16), (unsigned)iz | ((unsigned)box << 16));
  w.td_out[slot] = make_float4(tMx, tMy, tMz, dx);
  w.dyz_out[slot] = make_float2(dy, dz);
#pragma unroll
  for (int j = 0; j < (NBT > 0 ? NBT : CRASH_MAX_BINS); ++j) {
    if (NBT == 0 && j >= nb) break;
    w.N_out[(int64_t)j * w.cap + slot] = N[j];
  }
}

// ------------------------------------------------------------------ emission
template <int NBT, bool HE, bool HEAT>
__global__ void __launch_bounds__(256) k_emit_mixed(StepArgs a, BinTables t, WFArgs w, int64_t g0,
                                                   int64_t n, int S) {
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const uint32_t step = (uint32_t)*a.step_dev;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  Tally tl{0, 0, 0, 0, 0};
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    int b = -1;
    bool alive = false;
    int ix = 0, iy = 0, iz = 0;
    float tMx = 0.f, tMy = 0.f, tMz = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    long long N[NBT > 0 ? NBT : CRASH_MAX_BINS];
    if (i < n) {
      const int64_t gid = g0 + i;
      b = box_of_packet(a.boxes, a.n_boxes, gid);
      const BoxMeta* M = a.boxes + b;
      const int64_t local = gid - M->pkt_off;
      const uint32_t W = M->win_hi - M->win_lo;
      const int s_local = (int)(local / W);
      const uint32_t p = M->win_lo + (uint32_t)(local - (int64_t)s_local * W);
      const int s = M->src_off + s_local;
      double dx, dy, dz;
      if (!iso_direction(M->seed, step, (uint32_t)s_local, p, dx, dy, dz)) {
        atomicOr(a.err, ERR_DIRECTION);
      } else {
        for (int j = 0; j < nb; ++j) {
          const long long base_c = a.src_base[(int64_t)s * nb + j];
          const long long rem = a.src_rem[(int64_t)s * nb + j];
          N[j] = base_c + ((long long)p < rem ? 1 : 0);
          tl.emitted += (unsigned long long)N[j];
        }
        tl.packets += 1;
        const double px = a.src_pos[3 * s], py = a.src_pos[3 * s + 1], pz = a.src_pos[3 * s + 2];
        ix = (int)floor(px); iy = (int)floor(py); iz = (int)floor(pz);
        // distances to the first faces, formed in FP64 then rounded once
        tMx = dx > 0 ? (float)(((double)(ix + 1) - px) / dx) : (dx < 0 ? (float)(((double)ix - px) / dx) : INFINITY);
        tMy = dy > 0 ? (float)(((double)(iy + 1) - py) / dy) : (dy < 0 ? (float)(((double)iy - py) / dy) : INFINITY);
        tMz = dz > 0 ? (float)(((double)(iz + 1) - pz) / dz) : (dz < 0 ? (float)(((double)iz - pz) / dz) : INFINITY);
        fx = (float)dx; fy = (float)dy; fz = (float)dz;
        const int r = trace_mixed<NBT, HE, HEAT>(ix, iy, iz, tMx, tMy, tMz, fx, fy, fz, N, M, a, t,
                                                 nb, S, tl);
        if (r == ESCAPED) {
          for (int j = 0; j < nb; ++j) tl.escaped += (unsigned long long)N[j];
        }
        alive = (r == ALIVE);
      }
    }
    const long long slot = append_slot(alive, w.count_out);
    if (alive) {
      if (slot >= w.cap) atomicOr(a.err, ERR_QUEUE);
      else store_packet<NBT>(w, slot, ix, iy, iz, b, tMx, tMy, tMz, fx, fy, fz, N, nb);
    }
    flush_warp(a, b, tl);
  }
}

// ------------------------------------------------------------------ passes
template <int NBT, bool HE, bool HEAT>
__global__ void __launch_bounds__(256) k_pass_mixed(StepArgs a, BinTables t, WFArgs w, int S) {
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const int64_t n = (int64_t)*w.count_in;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  Tally tl{0, 0, 0, 0, 0};
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    int b = -1;
    bool alive = false;
    int ix = 0, iy = 0, iz = 0;
    float tMx = 0.f, tMy = 0.f, tMz = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    long long N[NBT > 0 ? NBT : CRASH_MAX_BINS];
    if (i < n) {
      const uint2 cb = w.cb_in[i];
      const float4 td = w.td_in[i];
      const float2 dd = w.dyz_in[i];
      ix = (int)(cb.x & 0xFFFFu); iy = (int)(cb.x >> 16);
      iz = (int)(cb.y & 0xFFFFu); b = (int)(cb.y >> 16);
      tMx = td.x; tMy = td.y; tMz = td.z; fx = td.w; fy = dd.x; fz = dd.y;
#pragma unroll
      for (int j = 0; j < (NBT > 0 ? NBT : CRASH_MAX_BINS); ++j) {
        if (NBT == 0 && j >= nb) break;
        N[j] = w.N_in[(int64_t)j * w.cap + i];
      }
      const BoxMeta* M = a.boxes + b;
      const int r = trace_mixed<NBT, HE, HEAT>(ix, iy, iz, tMx, tMy, tMz, fx, fy, fz, N, M, a, t,
                                               nb, S, tl);
      if (r == ESCAPED) {
        for (int j = 0; j < nb; ++j) tl.escaped += (unsigned long long)N[j];
      }
      alive = (r == ALIVE);
    }
    const long long slot = append_slot(alive, w.count_out);
    if (alive) {
      if (slot >= w.cap) atomicOr(a.err, ERR_QUEUE);
      else store_packet<NBT>(w, slot, ix, iy, iz, b, tMx, tMy, tMz, fx, fy, fz, N, nb);
    }
    flush_warp(a, b, tl);
  }
}

// ------------------------------------------------------------------ re-sort
__device__ __forceinline__ unsigned spread3(unsigned v) {   // 10 bits -> every third bit
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void k_sort_keys(StepArgs a, WFArgs w, unsigned* key, unsigned* rank, unsigned* bcount) {
  const int64_t n = (int64_t)*w.count_in;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const unsigned full = 0xFFFFFFFFu;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    unsigned k = 0xFFFFFFFFu;
    if (i < n) {
      const uint2 cb = w.cb_in[i];
      const float4 td = w.td_in[i];
      const float2 dd = w.dyz_in[i];
      const unsigned ix = cb.x & 0xFFFFu, iy = cb.x >> 16, iz = cb.y & 0xFFFFu, b = cb.y >> 16;
      const unsigned oct = (td.w < 0.f ? 1u : 0u) | (dd.x < 0.f ? 2u : 0u) | (dd.y < 0.f ? 4u : 0u);
      const unsigned mort = spread3(ix >> 3) | (spread3(iy >> 3) << 1) | (spread3(iz >> 3) << 2);
      k = (unsigned)a.boxes[b].bucket_off + ((mort << 3) | oct);
      key[i] = k;
    }
    // packets of a warp that share a key take one atomic
    const unsigned peers = __match_any_sync(full, k);
    if (i < n) {
      const int lane = threadIdx.x & 31;
      const int leader = __ffs(peers) - 1;
      unsigned r0 = 0;
      if (lane == leader) r0 = atomicAdd(&bcount[k], (unsigned)__popc(peers));
      r0 = __shfl_sync(peers, r0, leader);
      rank[i] = r0 + __popc(peers & ((1u << lane) - 1u));
    }
  }
}

// exclusive scan of bcount into boff: 4096 keys per block, block sums, add
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* sh, unsigned* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const unsigned warp_base = wid > 0 ? sh[wid - 1] : 0u;
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_base + x - v;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(const unsigned* in, unsigned* out,
                                                      unsigned* bsum, int64_t n) {
  __shared__ unsigned sh[32];
  const int64_t base = (int64_t)blockIdx.x * 4096 + threadIdx.x * 4;
  unsigned v[4], s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  unsigned tot;
  unsigned ex = block_excl_scan(s, sh, &tot);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_sums(unsigned* bsum, int nblocks) {
  __shared__ unsigned sh[32];
  const unsigned v = threadIdx.x < (unsigned)nblocks ? bsum[threadIdx.x] : 0u;
  unsigned tot;
  const unsigned ex = block_excl_scan(v, sh, &tot);
  if (threadIdx.x < (unsigned)nblocks) bsum[threadIdx.x] = ex;
}

__global__ void k_scan_add(unsigned* out, const unsigned* bsum, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += bsum[i >> 12];
}

template <int NBT>
__global__ void k_scatter(WFArgs w, const unsigned* key, const unsigned* rank, const unsigned* boff,
                          int nb, int* err) {
  const int64_t n = (int64_t)*w.count_in;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) *w.count_out = (unsigned)n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t d = (int64_t)boff[key[i]] + rank[i];
    if (d >= n) { atomicOr(err, ERR_QUEUE); continue; }
    w.cb_out[d] = w.cb_in[i];
    w.td_out[d] = w.td_in[i];
    w.dyz_out[d] = w.dyz_in[i];
#pragma unroll
    for (int j = 0; j < (NBT > 0 ? NBT : CRASH_MAX_BINS); ++j) {
      if (NBT == 0 && j >= nb) break;
      w.N_out[(int64_t)j * w.cap + d] = w.N_in[(int64_t)j * w.cap + i];
    }
  }
}

__global__ void k_check_drained(const unsigned* count, int* err) {
  if (*count != 0u) atomicOr(err, ERR_WATCHDOG);
}

WFArgs wf_args(WF* wf, int in) {
  WFArgs w;
  const int out = 1 - in;
  w.cb_in = wf->cb[in]; w.td_in = wf->td[in]; w.dyz_in = wf->dyz[in]; w.N_in = wf->N[in];
  w.cb_out = wf->cb[out]; w.td_out = wf->td[out]; w.dyz_out = wf->dyz[out]; w.N_out = wf->N[out];
  w.count_in = wf->count + in;
  w.count_out = wf->count + out;
  w.cap = wf->cap;
  return w;
}

int g_num_sms = 0;

int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 152;
  }
  return g_num_sms;
}

template <int NBT, bool HE, bool HEAT>
int run_mixed(const StepArgs& a, const BinTables& t, const crash_run_opts& o, WF* wf, int max_iter,
              cudaStream_t s, EventPairs* ev, int* ev_used) {
  int launches = 0;
  const int block = o.block_size > 0 ? o.block_size : 256;
  const int persistent = num_sms() * (2048 / block);
  auto tic = [&]() {
    if (!ev) return;
    if (*ev_used >= (int)ev->size()) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      ev->push_back({e0, e1});
    }
    cudaEventRecord((*ev)[*ev_used].first, s);
  };
  auto toc = [&]() {
    if (!ev) return;
    cudaEventRecord((*ev)[*ev_used].second, s);
    (*ev_used)++;
  };
  if (a.total_packets <= 0) return 0;
  if (!o.wavefront || wf->cap == 0) {
    // one thread per packet, traced to the end
    WFArgs w = wf_args(wf, 0);
    int64_t blocks = (a.total_packets + block - 1) / block;
    if (blocks > (int64_t)1 << 30) blocks = (int64_t)1 << 30;
    tic();
    k_emit_mixed<NBT, HE, HEAT><<<(unsigned)blocks, block, 0, s>>>(a, t, w, 0, a.total_packets, max_iter);
    toc();
    return 1;
  }
  const int S = o.seg_per_iter > 0 ? o.seg_per_iter : 64;
  const int R = o.resort_interval == 0 ? 2 : o.resort_interval;
  const int passes = (max_iter + S - 1) / S;
  const int nscan = (int)((wf->n_keys + 4095) / 4096);
  for (int64_t g0 = 0; g0 < a.total_packets; g0 += wf->cap) {
    const int64_t n = std::min<int64_t>(wf->cap, a.total_packets - g0);
    int cur = 0;
    cudaMemsetAsync(wf->count, 0, 4 * sizeof(unsigned), s);
    {
      WFArgs w = wf_args(wf, 1);     // emission writes survivors into buffer 0
      w.count_out = wf->count + 0;
      w.cb_out = wf->cb[0]; w.td_out = wf->td[0]; w.dyz_out = wf->dyz[0]; w.N_out = wf->N[0];
      int64_t blocks = (n + block - 1) / block;
      if (blocks > persistent * 4) blocks = persistent * 4;
      tic();
      k_emit_mixed<NBT, HE, HEAT><<<(unsigned)blocks, block, 0, s>>>(a, t, w, g0, n, S);
      toc();
      ++launches;
    }
    for (int p = 1; p < passes; ++p) {
      if (R > 0 && (p % R) == 0) {
        WFArgs w = wf_args(wf, cur);
        cudaMemsetAsync(wf->bcount, 0, sizeof(unsigned) * wf->n_keys, s);
        k_sort_keys<<<persistent, block, 0, s>>>(a, w, wf->key, wf->rank, wf->bcount);
        k_scan_blocks<<<nscan, 1024, 0, s>>>(wf->bcount, wf->boff, wf->bsum, wf->n_keys);
        k_scan_sums<<<1, 1024, 0, s>>>(wf->bsum, nscan);
        k_scan_add<<<(unsigned)((wf->n_keys + 255) / 256), 256, 0, s>>>(wf->boff, wf->bsum, wf->n_keys);
        k_scatter<NBT><<<persistent, block, 0, s>>>(w, wf->key, wf->rank, wf->boff, t.n_bins, a.err);
        launches += 5;
        cur = 1 - cur;
      }
      WFArgs w = wf_args(wf, cur);
      cudaMemsetAsync(w.count_out, 0, sizeof(unsigned), s);
      tic();
      k_pass_mixed<NBT, HE, HEAT><<<persistent, block, 0, s>>>(a, t, w, S);
      toc();
      ++launches;
      cur = 1 - cur;
    }
    k_check_drained<<<1, 1, 0, s>>>(wf->count + cur, a.err);
    ++launches;
  }
  return launches;
}

}  // namespace

int launch_trace_mixed(const StepArgs& a, const BinTables& t, const crash_run_opts& o, void* wfp,
                       int max_iter, cudaStream_t s, EventPairs* ev, int* ev_used) {
  WF* wf = (WF*)wfp;
  const bool he = a.any_he != 0, heat = a.any_heat != 0;
  int r;
  if (t.n_bins == 1) {
    if (he) r = heat ? run_mixed<1, true, true>(a, t, o, wf, max_iter, s, ev, ev_used)
                     : run_mixed<1, true, false>(a, t, o, wf, max_iter, s, ev, ev_used);
    else r = heat ? run_mixed<1, false, true>(a, t, o, wf, max_iter, s, ev, ev_used)
                  : run_mixed<1, false, false>(a, t, o, wf, max_iter, s, ev, ev_used);
  } else if (t.n_bins == 8) {
    if (he) r = heat ? run_mixed<8, true, true>(a, t, o, wf, max_iter, s, ev, ev_used)
                     : run_mixed<8, true, false>(a, t, o, wf, max_iter, s, ev, ev_used);
    else r = heat ? run_mixed<8, false, true>(a, t, o, wf, max_iter, s, ev, ev_used)
                  : run_mixed<8, false, false>(a, t, o, wf, max_iter, s, ev, ev_used);
  } else {
    if (he) r = heat ? run_mixed<0, true, true>(a, t, o, wf, max_iter, s, ev, ev_used)
                     : run_mixed<0, true, false>(a, t, o, wf, max_iter, s, ev, ev_used);
    else r = heat ? run_mixed<0, false, true>(a, t, o, wf, max_iter, s, ev, ev_used)
                  : run_mixed<0, false, false>(a, t, o, wf, max_iter, s, ev, ev_used);
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  return r;
}

void* wavefront_create(int64_t cap, int64_t n_keys, int nb, cudaError_t* err) {
  WF* w = new WF();
  w->cap = cap;
  w->nb = nb;
  w->n_keys = n_keys;
  cudaError_t e = cudaMalloc(&w->count, 4 * sizeof(unsigned));
  if (e == cudaSuccess && cap > 0) {
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaMalloc(&w->cb[b], sizeof(uint2) * cap);
      if (e == cudaSuccess) e = cudaMalloc(&w->td[b], sizeof(float4) * cap);
      if (e == cudaSuccess) e = cudaMalloc(&w->dyz[b], sizeof(float2) * cap);
      if (e == cudaSuccess) e = cudaMalloc(&w->N[b], sizeof(long long) * cap * nb);
    }
    if (e == cudaSuccess) e = cudaMalloc(&w->key, sizeof(unsigned) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&w->rank, sizeof(unsigned) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&w->bcount, sizeof(unsigned) * n_keys);
    if (e == cudaSuccess) e = cudaMalloc(&w->boff, sizeof(unsigned) * n_keys);
    if (e == cudaSuccess) e = cudaMalloc(&w->bsum, sizeof(unsigned) * 1024);
  }
  if (err) *err = e;
  if (e != cudaSuccess) {
    wavefront_destroy(w);
    return nullptr;
  }
  return w;
}

void wavefront_destroy(void* p) {
  WF* w = (WF*)p;
  if (!w) return;
  void* ptrs[] = {w->count, w->key, w->rank, w->bcount, w->boff, w->bsum,
                  w->cb[0], w->cb[1], w->td[0], w->td[1], w->dyz[0], w->dyz[1], w->N[0], w->N[1]};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete w;
}

int64_t wavefront_capacity(void* p) { return p ? ((WF*)p)->cap : 0; }
