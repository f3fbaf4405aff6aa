// k_mixed.cu -- mixed-precision transport: FP32 traversal, segment lengths
// and attenuation, exact int64 photon bookkeeping, FP64 only for the
// direction draw (so that every packet flies along the same direction as in
// the FP64 form).
//
// Per crossed cell and bin j (Sec. 2, Eq. 1): tau_j = l sum_s n_s sigma_s,j;
// the absorbed count A_j = rint(N_j (1 - e^-tau_j)) <= N_j is an integer and
// N' = N - A, so the photon budget stays exact; the species split (Sec. 2) and the
// heating energy are accumulated in FP32 over the bins and rounded once per
// cell, H I taking the remainder.
//
// Two launch shapes:
//   * one thread per packet (opts.wavefront = 0): emit and trace to the end;
//   * wavefront (default): the emission kernel writes every packet to a
//     device queue; pass kernels (persistent, grid-stride over the live
//     count held in device memory) advance the queue S steps at a time until
//     it is empty.  Every
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

// Packet records: array of structures, one record per packet (layout at
// store_record).
struct WF {
  int64_t cap = 0;
  int nb = 0;
  int rs = 0;                            // record size in bytes
  char* rec[2] = {nullptr, nullptr};
  unsigned* count = nullptr;             // [4]: live counts of buffers 0 and 1
  unsigned* key = nullptr;               // [cap] sort key of each written record
  unsigned* rank = nullptr;              // [cap] its rank among equal keys
  unsigned* perm = nullptr;              // [cap] sorted position -> record index
  unsigned* bcount = nullptr;            // [n_keys]
  unsigned* boff = nullptr;              // [n_keys]
  unsigned* bsum = nullptr;              // [1024]
  uint2* items = nullptr;                // work items of a tile pass (tile, first position)
  unsigned* gsync = nullptr;             // [2] grid barrier of the persistent launch
  int64_t n_keys = 0;
};

struct WFArgs {
  const char* rec_in;
  char* rec_out;
  const unsigned* count_in;
  unsigned* count_out;
  const unsigned* perm;      // non-null: read record perm[j] at position j
  unsigned* key;             // non-null: record the sort key and rank of every survivor
  unsigned* rank;
  unsigned* bcount;
  int rs;
  int tile;                  // keys of 16^3-cell tiles (tile passes) instead of 8^3 buckets
  int curve;                 // 0: Morton order of the buckets, 1: Hilbert order
  int64_t cap;
  unsigned* work;            // pass kernels: counter of the queue positions handed out
  unsigned* work_next;       // the next pass's counter, cleared by this pass
};

// Blocks of a pass take the next blockDim.x packets of the queue as they
// finish: walks differ in length, and a fixed grid stride leaves blocks idle
// at the end of the pass while a few finish theirs.  Returns the first
// position of the block's packets (>= n: the queue is exhausted).
__device__ __forceinline__ int64_t next_block_packets(unsigned* work) {
  __shared__ unsigned s_base;
  __syncthreads();                   // every thread has read the previous s_base
  if (threadIdx.x == 0) s_base = atomicAdd(work, (unsigned)blockDim.x);
  __syncthreads();
  return (int64_t)s_base;
}

struct Tally {
  unsigned long long emitted, absorbed, escaped;
  unsigned crossings, packets;       // per thread between flushes: far below 2^32
};

__device__ __forceinline__ void flush_warp(const StepArgs& a, int b, Tally& t) {
  const unsigned full = 0xFFFFFFFFu;
  const int b0 = __shfl_sync(full, b, 0);
  if (__all_sync(full, b == b0 || b < 0)) {
    t.emitted = warp_sum_u64(t.emitted);
    t.absorbed = warp_sum_u64(t.absorbed);
    t.escaped = warp_sum_u64(t.escaped);
    const unsigned long long cr = warp_sum_u64(t.crossings);
    const unsigned long long pk = warp_sum_u64(t.packets);
    if ((threadIdx.x & 31) == 0 && b0 >= 0) {
      unsigned long long* g = a.budget + b0 * 8;
      if (t.emitted) atomicAdd(g + 0, t.emitted);
      if (t.absorbed) atomicAdd(g + 1, t.absorbed);
      if (t.escaped) atomicAdd(g + 2, t.escaped);
      if (cr) atomicAdd(g + 3, cr);
      if (pk) atomicAdd(g + 4, pk);
    }
  } else if (b >= 0) {
    unsigned long long* g = a.budget + b * 8;
    if (t.emitted) atomicAdd(g + 0, t.emitted);
    if (t.absorbed) atomicAdd(g + 1, t.absorbed);
    if (t.escaped) atomicAdd(g + 2, t.escaped);
    if (t.crossings) atomicAdd(g + 3, (unsigned long long)t.crossings);
    if (t.packets) atomicAdd(g + 4, (unsigned long long)t.packets);
  }
  t = Tally{0, 0, 0, 0u, 0u};
}

// FP32 <-> integer conversions without the hardware 64-bit conversions,
// which on this GPU issue to the narrow FP64 pipe.
// rint(x) for x in [0, 2^63), round half to even, from two 32-bit
// conversions: hi = floor(x / 2^32) and the rest x - hi 2^32, which the fma
// gives exactly (below 2^32 the rest is x itself; above it x is an integer
// whose low part fits the 24-bit significand, or hi holds all of x).
__device__ __forceinline__ long long float_to_ll(float x) {
  const unsigned hi = __float2uint_rz(x * 2.3283064365386963e-10f);
  const unsigned lo = __float2uint_rn(fmaf(-__uint2float_rn(hi), 4294967296.0f, x));
  return (long long)(((unsigned long long)hi << 32) | lo);
}

// rint of the three per-cell shares x1, x2, xh (each at most about the
// cell's absorbed total Au): with Au below 2^31 all three fit the 32-bit
// conversion, which is then the whole rounding
__device__ __forceinline__ void round_shares(long long Au, float x1, float x2, float xh, long long& a1,
                                             long long& a2, long long& h) {
  if ((unsigned long long)Au < 0x80000000ull) {
    a1 = (long long)__float2uint_rn(x1);
    a2 = (long long)__float2uint_rn(x2);
    h = (long long)__float2uint_rn(xh);
  } else {
    a1 = float_to_ll(x1);
    a2 = float_to_ll(x2);
    h = float_to_ll(xh);
  }
}

// (1 - exp(-tau)) / tau for 0 <= tau <= 0.5: a degree-5 polynomial fitted
// for the smallest largest relative error on [0, 0.5] (Lawson's iteration
// on 4000 Chebyshev-spaced points).  With its coefficients rounded to FP32
// the polynomial is within 7e-9 of the function; evaluated in FP32 by
// Horner's rule the result is within 5.4e-8 (the Taylor series to tau^7
// gave 5.7e-8 with two more steps).  tests/test_series_poly.py checks both.
#define CRASH_AOT_C0 1.0f
#define CRASH_AOT_C1 -0.4999998211860657f
#define CRASH_AOT_C2 0.16666224598884583f
#define CRASH_AOT_C3 -0.041629090905189514f
#define CRASH_AOT_C4 0.008187386207282543f
#define CRASH_AOT_C5 -0.0011216348502784967f
__device__ __forceinline__ float absorbed_over_tau(float tau) {
  float p = CRASH_AOT_C5;
  p = fmaf(p, tau, CRASH_AOT_C4);
  p = fmaf(p, tau, CRASH_AOT_C3);
  p = fmaf(p, tau, CRASH_AOT_C2);
  p = fmaf(p, tau, CRASH_AOT_C1);
  p = fmaf(p, tau, CRASH_AOT_C0);
  return p;
}

// rint(x) for x in [0, 2^32), round half to even
__device__ __forceinline__ unsigned float_to_u32(float x) {
  if (x < 8388608.0f) return __float_as_uint(x + 8388608.0f) - 0x4B000000u;
  return __float2uint_rn(x);
}

// Absorbed count of one bin of content m (in the packet's units): for
// tau < 0.5 round m (1 - e^-tau), else round the transmitted m e^-tau and
// take the difference, so that the smaller of the two parts always carries
// ~1e-7 relative error.  q is the absorbed count divided by tau in FP32: the
// share of species s is q k_s.
__device__ __forceinline__ unsigned absorb(unsigned m, float tau, float& q) {
  const float Nf = __uint2float_rn(m);
  if (tau < 0.5f) {
    q = Nf * absorbed_over_tau(tau);
    const unsigned A = float_to_u32(q * tau);
    return A > m ? m : A;
  }
  const float T = Nf * expf(-tau);
  q = (Nf - T) * __fdividef(1.0f, tau);
  unsigned Np = float_to_u32(T);
  Np = Np > m ? m : Np;
  return m - Np;
}

// Packet content: per bin a 32-bit count m_j in units of 2^e photon quanta
// (e >= 0 is the packet's exponent), so N_j = m_j 2^e exactly.
template <int NBT>
struct Content {
  unsigned m[NBT > 0 ? NBT : CRASH_MAX_BINS];
  int e;
  __device__ __forceinline__ unsigned long long total(int nb) const {
    unsigned long long t = 0;
    for (int j = 0; j < nb; ++j) t += m[j];
    return t << e;
  }
};

// Two FP32 lanes in one 64-bit register for the packed f32x2 arithmetic of
// this GPU (fma/mul/add on both lanes in one instruction).  Each lane is
// rounded exactly as the scalar instruction, so a pair of bins done packed
// gives the same bits as the two bins done one by one.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_split(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

enum { ALIVE = 0, ABSORBED = 1, ESCAPED = 2 };

// One bin's absorbed count once its optical depth tau and the series value
// q = Nf (1 - e^-tau)/tau (tau < 0.5) are known: the same rounding as
// absorb(), with the transmitted part taken for tau >= 0.5 (q replaced).
__device__ __forceinline__ unsigned absorb_lane(unsigned m, float Nf, float tau, float& q) {
  if (tau < 0.5f) {
    const unsigned A = __float2uint_rn(q * tau);
    return A > m ? m : A;
  }
  const float T = Nf * expf(-tau);
  q = (Nf - T) * __fdividef(1.0f, tau);
  unsigned Np = __float2uint_rn(T);
  Np = Np > m ? m : Np;
  return m - Np;
}

// cell_attenuate for an even number of bins, two bins per packed
// instruction: the optical depths, the series, the absorbed counts and the
// species and heating sums of a bin pair in f32x2; the rounding to counts
// per bin.  Gives the same bits as the scalar form (whose sums run over the
// even and the odd bins separately, as the two lanes do).
//
// The species and heating sums factor the segment's optical depth per
// species out of the bin sum: the share of species s in bin j is
// q_j t_s sigma_s,j (q_j the absorbed count over tau_j, t_s = l n_s), so the
// cell's He I share is t_HeI sum_j q_j sigma_HeI,j and its heating
// sum_s t_s sum_j q_j (sigma w)_s,j; per bin pair that is one packed fma per
// sum.
//
// THIN: every bin of the cell has tau < 0.5 (known from one bound for the
// whole cell), so every bin takes the series and A = rint(m (1 - e^-tau))
// needs no clamp: it is at most 0.4 m + 1/2, below m for m >= 1, so a bin
// that held photons still holds some and the packet's liveness is unchanged
// (left is not recomputed).
template <int NBT, bool HE, bool HEAT, bool THIN>
__device__ __forceinline__ void attenuate_bins_x2(const f32x2 tHI2, const f32x2 tHeI2, const f32x2 tHeII2,
                                                  Content<NBT>& c, const BinTables& t,
                                                  unsigned long long& At, unsigned& left, f32x2& g1,
                                                  f32x2& g2, f32x2& h0, f32x2& h1, f32x2& h2) {
  if (!THIN) left = 0;
#pragma unroll
  for (int j = 0; j < NBT; j += 2) {
    const f32x2 s0 = f2(t.sigma32[0][j], t.sigma32[0][j + 1]);
    f32x2 tau = f2_mul(tHI2, s0);
    f32x2 s1 = 0ull, s2 = 0ull;
    if (HE) {
      s1 = f2(t.sigma32[1][j], t.sigma32[1][j + 1]);
      s2 = f2(t.sigma32[2][j], t.sigma32[2][j + 1]);
      tau = f2_fma(tHeII2, s2, f2_fma(tHeI2, s1, tau));
    }
    const unsigned m0 = c.m[j], m1 = c.m[j + 1];
    const float N0 = __uint2float_rn(m0), N1 = __uint2float_rn(m1);
    // (1 - e^-tau)/tau by the same Horner steps as absorbed_over_tau
    f32x2 p = f2(CRASH_AOT_C5, CRASH_AOT_C5);
    p = f2_fma(p, tau, f2(CRASH_AOT_C4, CRASH_AOT_C4));
    p = f2_fma(p, tau, f2(CRASH_AOT_C3, CRASH_AOT_C3));
    p = f2_fma(p, tau, f2(CRASH_AOT_C2, CRASH_AOT_C2));
    p = f2_fma(p, tau, f2(CRASH_AOT_C1, CRASH_AOT_C1));
    p = f2_fma(p, tau, f2(CRASH_AOT_C0, CRASH_AOT_C0));
    f32x2 q2 = f2_mul(f2(N0, N1), p);
    // a bin with no photons or no optical depth absorbs nothing and adds
    // nothing below (q = 0 or sigma = 0), as when the scalar form skips it
    unsigned A0, A1;
    if (THIN) {
      float qt0, qt1;
      f2_split(f2_mul(q2, tau), qt0, qt1);
      A0 = __float2uint_rn(qt0);
      A1 = __float2uint_rn(qt1);
    } else {
      float tau0, tau1, q0, q1;
      f2_split(tau, tau0, tau1);
      f2_split(q2, q0, q1);
      A0 = absorb_lane(m0, N0, tau0, q0);
      A1 = absorb_lane(m1, N1, tau1, q1);
      q2 = f2(q0, q1);
    }
    c.m[j] = m0 - A0;
    c.m[j + 1] = m1 - A1;
    At += A0;
    At += A1;
    if (!THIN) left |= (m0 - A0) | (m1 - A1);
    if (HE) {
      g1 = f2_fma(q2, s1, g1);
      g2 = f2_fma(q2, s2, g2);
    }
    if (HEAT) {
      h0 = f2_fma(q2, f2(t.sw32[0][j], t.sw32[0][j + 1]), h0);
      if (HE) {
        h1 = f2_fma(q2, f2(t.sw32[1][j], t.sw32[1][j + 1]), h1);
        h2 = f2_fma(q2, f2(t.sw32[2][j], t.sw32[2][j + 1]), h2);
      }
    }
  }
}

// the sum of the two lanes of a pair
__device__ __forceinline__ float f2_sum(f32x2 v) {
  float lo, hi;
  f2_split(v, lo, hi);
  return lo + hi;
}

// The cell's species and heating shares from the per-species bin sums (in
// the packet's units), scaled to photon quanta and rounded once: He I and
// He II clamped to the absorbed total, H I taking the rest.
template <bool HE, bool HEAT>
__device__ __forceinline__ void cell_shares(unsigned long long At, int e, float tHI, float tHeI, float tHeII,
                                            float G1, float G2, float H0, float H1, float H2,
                                            long long& dHI, long long& dHeI, long long& dHeII,
                                            long long& dE) {
  long long a1 = 0, a2 = 0, h = 0;
  const long long Au = (long long)(At << e);
  if (At) {
    const float unit = __uint_as_float((unsigned)(127 + e) << 23);
    const float fHeI = HE ? tHeI * G1 : 0.f, fHeII = HE ? tHeII * G2 : 0.f;
    const float fheat = HEAT ? (HE ? fmaf(tHeII, H2, fmaf(tHeI, H1, tHI * H0)) : tHI * H0) : 0.f;
    round_shares(Au, fHeI * unit, fHeII * unit, fheat * unit, a1, a2, h);
    if (!HE) a1 = a2 = 0;
    if (!HEAT) h = 0;
    // He shares above the cell's total only by rounding: clamp then (the
    // clamps change nothing when the two fit)
    if (HE && (unsigned long long)a1 + (unsigned long long)a2 > (unsigned long long)Au) {
      a1 = a1 > Au ? Au : a1;
      a2 = a2 > Au - a1 ? Au - a1 : a2;
    }
  }
  dHeI = a1;
  dHeII = a2;
  dHI = Au - a1 - a2;
  dE = h;
}

// left: on entry, nonzero if some bin holds photons; on return, the same
// after the cell
template <int NBT, bool HE, bool HEAT>
__device__ __forceinline__ long long cell_attenuate_x2(float seg, float dl, float4 ab, Content<NBT>& c,
                                                       const BinTables& t, long long& dHI,
                                                       long long& dHeI, long long& dHeII, long long& dE,
                                                       unsigned& left) {
  static_assert(NBT >= 2 && NBT % 2 == 0, "bin pairs");
  const float l = seg * dl;
  const float tHI = l * ab.x, tHeI = l * ab.y, tHeII = l * ab.z;
  const f32x2 tHI2 = f2(tHI, tHI), tHeI2 = f2(tHeI, tHeI), tHeII2 = f2(tHeII, tHeII);
  unsigned long long At = 0;
  f32x2 g1 = 0ull, g2 = 0ull, h0 = 0ull, h1 = 0ull, h2 = 0ull;
  // the optical depth of every bin is at most this bound, computed with the
  // largest cross sections in the same operation order (rounding is monotone)
  const float k0max = tHI * t.sigma32_max[0];
  const float tau_max = HE ? fmaf(tHeII, t.sigma32_max[2], fmaf(tHeI, t.sigma32_max[1], k0max)) : k0max;
  if (tau_max < 0.5f)
    attenuate_bins_x2<NBT, HE, HEAT, true>(tHI2, tHeI2, tHeII2, c, t, At, left, g1, g2, h0, h1, h2);
  else
    attenuate_bins_x2<NBT, HE, HEAT, false>(tHI2, tHeI2, tHeII2, c, t, At, left, g1, g2, h0, h1, h2);
  cell_shares<HE, HEAT>(At, c.e, tHI, tHeI, tHeII, f2_sum(g1), f2_sum(g2), f2_sum(h0), f2_sum(h1),
                        f2_sum(h2), dHI, dHeI, dHeII, dE);
  return (long long)(At << c.e);
}

// Attenuation and deposition in one crossed cell (Sec. 2, Eq. 1) for a
// segment of seg cells: updates the packet's bins and returns the absorbed
// total in photon quanta; the species and heating deposits of the cell come
// back in d* (quanta), left is nonzero while some bin holds photons.  The
// species and heating sums run over the even and the odd bins separately
// and are then added, as the two lanes of the packed form do.
template <int NBT, bool HE, bool HEAT>
__device__ __forceinline__ long long cell_attenuate(float seg, float dl, float4 ab, Content<NBT>& c,
                                                    int nb, const BinTables& t, long long& dHI,
                                                    long long& dHeI, long long& dHeII, long long& dE,
                                                    unsigned& left) {
  if constexpr (NBT >= 2 && NBT % 2 == 0)
    return cell_attenuate_x2<NBT, HE, HEAT>(seg, dl, ab, c, t, dHI, dHeI, dHeII, dE, left);
  const float l = seg * dl;
  const float tHI = l * ab.x, tHeI = l * ab.y, tHeII = l * ab.z;
  unsigned long long At = 0;
  left = 0;
  float g1[2] = {0.f, 0.f}, g2[2] = {0.f, 0.f}, h0[2] = {0.f, 0.f}, h1[2] = {0.f, 0.f}, h2[2] = {0.f, 0.f};
#pragma unroll
  for (int j = 0; j < (NBT > 0 ? NBT : CRASH_MAX_BINS); ++j) {
    if (NBT == 0 && j >= nb) break;
    float tau = tHI * t.sigma32[0][j];
    if (HE) tau = fmaf(tHeII, t.sigma32[2][j], fmaf(tHeI, t.sigma32[1][j], tau));
    unsigned mj = c.m[j];
    if (mj > 0u) {
      float q;
      const unsigned A = absorb(mj, tau, q);
      mj -= A;
      c.m[j] = mj;
      At += A;
      const int o = j & 1;
      if (HE) {
        g1[o] = fmaf(q, t.sigma32[1][j], g1[o]);
        g2[o] = fmaf(q, t.sigma32[2][j], g2[o]);
      }
      if (HEAT) {
        h0[o] = fmaf(q, t.sw32[0][j], h0[o]);
        if (HE) {
          h1[o] = fmaf(q, t.sw32[1][j], h1[o]);
          h2[o] = fmaf(q, t.sw32[2][j], h2[o]);
        }
      }
    }
    left |= mj;
  }
  cell_shares<HE, HEAT>(At, c.e, tHI, tHeI, tHeII, g1[0] + g1[1], g2[0] + g2[1], h0[0] + h0[1],
                        h1[0] + h1[1], h2[0] + h2[1], dHI, dHeI, dHeII, dE);
  return (long long)(At << c.e);
}

// Where a walk reads absorbers and adds deposits: the grid in global memory
// (gathers through L1, deposits reduced in L2) ...
//
// The four int64 deposits of a crossing are one 32-byte record, so they go
// to L2 as one bulk reduction (cp.reduce.async.bulk .add.u64) from a 32-byte
// slot of shared memory per thread instead of four separate reductions.
// Two slots alternate: a slot is rewritten only after the bulk operation
// issued from it two crossings earlier has read it.  Integer sums do not
// depend on their order, so the deposits are the same bits either way.
// Without a slot (stage == nullptr: more than kStageThreads threads, or a
// deposit array not aligned to 16 bytes) the thread uses plain reductions.
constexpr int kStageThreads = 256;

__device__ __forceinline__ void bulk_add_u64x4(unsigned long long* gdst, unsigned long long* slot,
                                               long long a0, long long a1, long long a2, long long e) {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
  reinterpret_cast<ulonglong2*>(slot)[0] = make_ulonglong2((unsigned long long)a0, (unsigned long long)a1);
  reinterpret_cast<ulonglong2*>(slot)[1] = make_ulonglong2((unsigned long long)a2, (unsigned long long)e);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(slot);
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], 32;"
               :: "l"(gdst), "r"(sa) : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// wait for every bulk operation this thread issued (reads of shared memory
// and the reductions in global memory)
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

struct GlobalCells {
  const float4* abs;
  unsigned long long* dep;
  int64_t coff;
  int nx, ny;
  unsigned long long* stage;     // this thread's two 32-byte slots (shared), or nullptr
  mutable int slot;
  __device__ __forceinline__ int64_t index(int ix, int iy, int iz) const {
    return coff + (ix + nx * (iy + ny * iz));
  }
  __device__ __forceinline__ float4 load(int64_t c, int, int, int) const { return __ldg(abs + c); }
  __device__ __forceinline__ void add(int64_t c, long long a0, long long a1, long long a2, long long e) const {
    unsigned long long* dp = dep + 4 * c;
    if (stage) {
      bulk_add_u64x4(dp, stage + 4 * slot, a0, a1, a2, e);
      slot ^= 1;
      return;
    }
    if (a0) atomicAdd(dp + 0, (unsigned long long)a0);
    if (a1) atomicAdd(dp + 1, (unsigned long long)a1);
    if (a2) atomicAdd(dp + 2, (unsigned long long)a2);
    if (e) atomicAdd(dp + 3, (unsigned long long)e);
  }
};

// ... or one 16^3-cell tile whose absorbers and deposits are both held in
// shared memory while the tile's packets cross it (cells indexed locally,
// lx + 16 (ly + 16 lz)); the deposits are int64 atomics in shared memory,
// one array of 4096 per species (so that lanes at different cells spread
// over the banks), and go to the grid once per work item
struct TileCells {
  const float4* sabs;              // shared, [16][16][16]
  unsigned long long* sdep;        // shared, [4][16][16][16]
  int x0, y0, z0;
  __device__ __forceinline__ int64_t index(int ix, int iy, int iz) const {
    return (ix - x0) + 16 * ((iy - y0) + 16 * (iz - z0));
  }
  __device__ __forceinline__ float4 load(int64_t c, int, int, int) const { return sabs[c]; }
  __device__ __forceinline__ void add(int64_t c, long long a0, long long a1, long long a2, long long e) const {
    if (a0) atomicAdd(sdep + c, (unsigned long long)a0);
    if (a1) atomicAdd(sdep + 4096 + c, (unsigned long long)a1);
    if (a2) atomicAdd(sdep + 8192 + c, (unsigned long long)a2);
    if (e) atomicAdd(sdep + 12288 + c, (unsigned long long)e);
  }
};

// Advance one packet by at most max_iter DDA steps.  tM* are the distances
// (in cells, along the ray) from the current point to the next x/y/z face;
// they are re-based at every step so that FP32 keeps their precision.  The
// walk does not depend on the attenuation, so the next cell's absorbers are
// requested before the current cell's bins are processed (one step of
// software pipelining hides most of the gather latency).  With TILE the walk
// also stops (alive) when it steps out of the box [tx0,tx0+ex) x ... .
// With PER, a box flagged periodic wraps the walk at its faces and ends it
// (ESCAPED) once the path trem (cells, the rest of c dt) is used up, the
// last segment cut there (Sec. 2 periodic boxes).  The photons the walk
// absorbed are counted once at its end, as the drop of the packet's content.
template <int NBT, bool HE, bool HEAT, bool TILE, bool PER, class Cells>
__device__ __forceinline__ int walk_steps(int& ix, int& iy, int& iz, float& tMx, float& tMy, float& tMz,
                                    const float dx, const float dy, const float dz, Content<NBT>& N,
                                    const BoxMeta* M, const Cells& cells, const BinTables& t,
                                    const int nb, const int max_iter, Tally& tl, int tx0 = 0,
                                    int ty0 = 0, int tz0 = 0, int ex = 0, int ey = 0, int ez = 0,
                                    float* trem = nullptr) {
  const int nx = M->nx, ny = M->ny, nz = M->nz;
  const bool per = PER && M->periodic;
  const float tDx = dx != 0.f ? 1.0f / fabsf(dx) : INFINITY;
  const float tDy = dy != 0.f ? 1.0f / fabsf(dy) : INFINITY;
  const float tDz = dz != 0.f ? 1.0f / fabsf(dz) : INFINITY;
  const int sx = dx > 0.f ? 1 : -1, sy = dy > 0.f ? 1 : -1, sz = dz > 0.f ? 1 : -1;
  const float dl = M->dlf;
  const bool heat_box = HEAT && !M->isothermal;
  if (max_iter <= 0) return ALIVE;
  unsigned left = 0;
#pragma unroll
  for (int j = 0; j < (NBT > 0 ? NBT : CRASH_MAX_BINS); ++j)
    if (NBT > 0 || j < nb) left |= N.m[j];
  // current segment
  float seg = fminf(tMx, fminf(tMy, tMz));
  int ax = (tMx <= tMy && tMx <= tMz) ? 0 : (tMy <= tMz ? 1 : 2);
  int64_t cell = cells.index(ix, iy, iz);
  float4 ab = cells.load(cell, ix, iy, iz);
  for (int it = 1;; ++it) {
    // step the walk into the next cell and request its absorbers
    const bool bx = ax == 0, by = ax == 1, bz = ax == 2;
    tMx = bx ? tDx : tMx - seg;
    tMy = by ? tDy : tMy - seg;
    tMz = bz ? tDz : tMz - seg;
    ix += bx ? sx : 0;
    iy += by ? sy : 0;
    iz += bz ? sz : 0;
    if (PER && per) {
      ix = ix < 0 ? nx - 1 : (ix >= nx ? 0 : ix);
      iy = iy < 0 ? ny - 1 : (iy >= ny ? 0 : iy);
      iz = iz < 0 ? nz - 1 : (iz >= nz ? 0 : iz);
    }
    const bool out = ((unsigned)ix >= (unsigned)nx) | ((unsigned)iy >= (unsigned)ny) |
                     ((unsigned)iz >= (unsigned)nz);
    const bool leave = TILE ? (((unsigned)(ix - tx0) >= (unsigned)ex) | ((unsigned)(iy - ty0) >= (unsigned)ey) |
                               ((unsigned)(iz - tz0) >= (unsigned)ez))
                            : out;
    float seg_n = 0.f;
    int ax_n = 0;
    int64_t cell_n = cell;
    float4 ab_n = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!leave) {
      seg_n = fminf(tMx, fminf(tMy, tMz));
      ax_n = (tMx <= tMy && tMx <= tMz) ? 0 : (tMy <= tMz ? 1 : 2);
      cell_n = cells.index(ix, iy, iz);
      ab_n = cells.load(cell_n, ix, iy, iz);
    }
    // periodic: the path left to the light-travel distance cuts the segment
    bool stop = false;
    if (PER && per) {
      stop = seg >= *trem;
      if (stop) seg = *trem;
      *trem -= seg;
    }
    // attenuate and deposit in the current cell
    if (seg > 0.f) {
      long long dHI, dHeI, dHeII, dE;
      const long long Atot = cell_attenuate<NBT, HE, HEAT>(seg, dl, ab, N, nb, t, dHI, dHeI, dHeII,
                                                           dE, left);
      if (Atot) cells.add(cell, dHI, dHeI, dHeII, heat_box ? dE : 0ll);
      tl.crossings += 1;
      if (left == 0) return ABSORBED;
    }
    if (PER && stop) return ESCAPED;
    if (out) return ESCAPED;
    if (TILE && leave) return ALIVE;
    if (it >= max_iter) return ALIVE;
    seg = seg_n;
    ax = ax_n;
    cell = cell_n;
    ab = ab_n;
  }
}

template <int NBT, bool HE, bool HEAT, bool TILE, bool PER, class Cells>
__device__ __forceinline__ int walk(int& ix, int& iy, int& iz, float& tMx, float& tMy, float& tMz,
                                    const float dx, const float dy, const float dz, Content<NBT>& N,
                                    const BoxMeta* M, const Cells& cells, const BinTables& t,
                                    const int nb, const int max_iter, Tally& tl, int tx0 = 0,
                                    int ty0 = 0, int tz0 = 0, int ex = 0, int ey = 0, int ez = 0,
                                    float* trem = nullptr) {
  tl.absorbed += N.total(nb);
  const int r = walk_steps<NBT, HE, HEAT, TILE, PER>(ix, iy, iz, tMx, tMy, tMz, dx, dy, dz, N, M, cells, t,
                                                     nb, max_iter, tl, tx0, ty0, tz0, ex, ey, ez, trem);
  tl.absorbed -= N.total(nb);
  return r;
}

// the walk over the grid in global memory
template <int NBT, bool HE, bool HEAT, bool PER = false>
__device__ __forceinline__ int trace_mixed(int& ix, int& iy, int& iz, float& tMx, float& tMy,
                                           float& tMz, const float dx, const float dy,
                                           const float dz, Content<NBT>& N, const BoxMeta* M,
                                           const StepArgs& a, const BinTables& t, const int nb,
                                           const int max_iter, Tally& tl, float* trem = nullptr) {
  __shared__ __align__(16) unsigned long long stage[kStageThreads * 8];
  const bool bulk = threadIdx.x < kStageThreads && ((uintptr_t)a.dep & 15u) == 0;
  GlobalCells cells{reinterpret_cast<const float4*>(a.abs32), a.dep, M->cell_off, M->nx, M->ny,
                    bulk ? stage + 8 * threadIdx.x : nullptr, 0};
  const int r = walk<NBT, HE, HEAT, false, PER>(ix, iy, iz, tMx, tMy, tMz, dx, dy, dz, N, M, cells, t,
                                                nb, max_iter, tl, 0, 0, 0, 0, 0, 0, trem);
  if (bulk) bulk_wait_all();
  return r;
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

// sort key: the packet's 8^3-cell bucket (16^3-cell tile for tile passes)
// along the Morton or Hilbert curve, then its direction octant
__device__ __forceinline__ unsigned sort_key(const BoxMeta* boxes, int box, int ix, int iy, int iz,
                                             float dx, float dy, float dz, int tile, int curve) {
  const unsigned oct = (dx < 0.f ? 1u : 0u) | (dy < 0.f ? 2u : 0u) | (dz < 0.f ? 4u : 0u);
  const int sh = tile ? 4 : 3;
  const BoxMeta& M = boxes[box];
  const unsigned pos = curve_key3((unsigned)ix >> sh, (unsigned)iy >> sh, (unsigned)iz >> sh,
                                  tile ? M.tile_bits : M.bucket_bits, curve != 0);
  const unsigned base = tile ? (unsigned)M.tile_off : (unsigned)M.bucket_off;
  return base + ((pos << 3) | oct);
}

// Packet records, RS bytes each (RS = 32 + 4 n_bins rounded up to 16 bytes,
// 64 for 8 bins):
//   [0,16)  float4 (tMx, tMy, tMz, dx)
//   [16,32) uint4  (ix | iy << 16, iz | box << 16 | e << 27, dy, dz)
//   [32, )  uint32 m[n_bins]
template <int NBT>
__device__ __forceinline__ void store_record(char* rec, int rs, long long slot, int ix, int iy, int iz,
                                             int box, float tMx, float tMy, float tMz, float dx,
                                             float dy, float dz, const Content<NBT>& c, int nb) {
  char* r = rec + (int64_t)rs * slot;
  *reinterpret_cast<float4*>(r) = make_float4(tMx, tMy, tMz, dx);
  *reinterpret_cast<uint4*>(r + 16) =
      make_uint4((unsigned)ix | ((unsigned)iy << 16),
                 (unsigned)iz | ((unsigned)box << 16) | ((unsigned)c.e << 27),
                 __float_as_uint(dy), __float_as_uint(dz));
  uint4* m4 = reinterpret_cast<uint4*>(r + 32);
#pragma unroll
  for (int j = 0; j < (NBT > 0 ? (NBT + 3) / 4 : CRASH_MAX_BINS / 4); ++j) {
    if (NBT == 0 && 4 * j >= nb) break;
    const int k = 4 * j;
    const int lim = NBT > 0 ? NBT : CRASH_MAX_BINS;
    m4[j] = make_uint4(c.m[k], (k + 1 < lim && k + 1 < nb) ? c.m[k + 1] : 0u,
                       (k + 2 < lim && k + 2 < nb) ? c.m[k + 2] : 0u,
                       (k + 3 < lim && k + 3 < nb) ? c.m[k + 3] : 0u);
  }
}

template <int NBT>
__device__ __forceinline__ void load_record(const char* rec, int rs, long long i, int& ix, int& iy,
                                            int& iz, int& box, float& tMx, float& tMy, float& tMz,
                                            float& dx, float& dy, float& dz, Content<NBT>& c, int nb) {
  const char* r = rec + (int64_t)rs * i;
  const float4 td = __ldcg(reinterpret_cast<const float4*>(r));
  const uint4 cd = __ldcg(reinterpret_cast<const uint4*>(r + 16));
  tMx = td.x; tMy = td.y; tMz = td.z; dx = td.w;
  ix = (int)(cd.x & 0xFFFFu); iy = (int)(cd.x >> 16);
  iz = (int)(cd.y & 0xFFFFu); box = (int)((cd.y >> 16) & 0x7FFu);
  c.e = (int)(cd.y >> 27);
  dy = __uint_as_float(cd.z); dz = __uint_as_float(cd.w);
  const uint4* m4 = reinterpret_cast<const uint4*>(r + 32);
  const int lim = NBT > 0 ? NBT : CRASH_MAX_BINS;
#pragma unroll
  for (int j = 0; j < (NBT > 0 ? (NBT + 3) / 4 : CRASH_MAX_BINS / 4); ++j) {
    if (NBT == 0 && 4 * j >= nb) break;
    const uint4 v = __ldcg(m4 + j);
    const int k = 4 * j;
    c.m[k] = v.x;
    if (k + 1 < lim) c.m[k + 1] = v.y;
    if (k + 2 < lim) c.m[k + 2] = v.z;
    if (k + 3 < lim) c.m[k + 3] = v.w;
  }
}

// Write the survivors of a warp: append slot, record, and (when the next
// pass reads in sorted order) the record's key and its rank among the
// records of that key (one atomic per group of equal keys in the warp).
template <int NBT>
__device__ __forceinline__ void write_survivor_to(const StepArgs& a, unsigned* count_out, int64_t cap, char* rec_out,
                                                  int rs, bool write_keys, unsigned* key, unsigned* rank,
                                                  unsigned* bcount, int tile, int curve, bool alive, int ix,
                                                  int iy, int iz, int box, float tMx, float tMy, float tMz,
                                                  float dx, float dy, float dz, const Content<NBT>& N, int nb) {
  const long long slot = append_slot(alive, count_out);
  bool ok = alive;
  if (alive && slot >= cap) {
    atomicOr(a.err, ERR_QUEUE);
    ok = false;
  }
  if (ok) store_record<NBT>(rec_out, rs, slot, ix, iy, iz, box, tMx, tMy, tMz, dx, dy, dz, N, nb);
  if (write_keys) {
    const unsigned k = ok ? sort_key(a.boxes, box, ix, iy, iz, dx, dy, dz, tile, curve) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
    if (ok) {
      const int lane = threadIdx.x & 31;
      const int leader = __ffs(peers) - 1;
      unsigned r0 = 0;
      if (lane == leader) r0 = atomicAdd(&bcount[k], (unsigned)__popc(peers));
      r0 = __shfl_sync(peers, r0, leader);
      key[slot] = k;
      rank[slot] = r0 + __popc(peers & ((1u << lane) - 1u));
    }
  }
}

template <int NBT>
__device__ __forceinline__ void write_survivor(const StepArgs& a, const WFArgs& w, bool alive, int ix,
                                               int iy, int iz, int box, float tMx, float tMy, float tMz,
                                               float dx, float dy, float dz, const Content<NBT>& N,
                                               int nb) {
  write_survivor_to<NBT>(a, w.count_out, w.cap, w.rec_out, w.rs, w.key != nullptr, w.key, w.rank, w.bcount,
                         w.tile, w.curve, alive, ix, iy, iz, box, tMx, tMy, tMz, dx, dy, dz, N, nb);
}

// ------------------------------------------------------------------ emission
// MINB = 3 keeps three 256-thread blocks resident per SM (at most 85
// registers); MINB = 4 caps the kernels at 64 registers for four.
// Emission of the packets [g0, g0 + n) of the launch, grid-stride over the
// calling grid: each is traced S steps (0: emission only) and, when the launch
// keeps a queue (S < max_steps_all), written to it with its sort key.
template <int NBT, bool HE, bool HEAT, bool PER>
__device__ __forceinline__ void emit_range(const StepArgs& a, const BinTables& t, const WFArgs& w, int64_t g0,
                                           int64_t n, int S, int max_steps_all) {
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const uint32_t step = (uint32_t)*a.step_dev;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  Tally tl{0, 0, 0, 0u, 0u};
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    int b = -1;
    bool alive = false;
    int ix = 0, iy = 0, iz = 0;
    float tMx = 0.f, tMy = 0.f, tMz = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    Content<NBT> N;
    N.e = 0;
    if (i < n) {
      const int64_t gid = g0 + i;
      b = box_of_packet(a.boxes, a.n_boxes, gid);
      const BoxMeta* M = a.boxes + b;
      const int64_t local = gid - M->pkt_off;
      const uint32_t W = M->win_hi - M->win_lo;
      const int s_local = (int)(local / W);
      const uint32_t p = M->win_lo + (uint32_t)(local - (int64_t)s_local * W);
      const int s = M->src_off + s_local;
      if (!iso_direction_f32(M->seed, step, (uint32_t)s_local, p, fx, fy, fz)) {
        atomicOr(a.err, ERR_DIRECTION);
      } else {
        // the packet's share of every bin in quanta, held as 32-bit counts
        // in units of 2^e (the low e bits, below 2^-31 of the packet, are not
        // emitted)
        unsigned long long q[NBT > 0 ? NBT : CRASH_MAX_BINS];
        unsigned long long qmax = 0;
        for (int j = 0; j < nb; ++j) {
          const long long base_c = a.src_base[(int64_t)s * nb + j];
          const long long rem = a.src_rem[(int64_t)s * nb + j];
          q[j] = (unsigned long long)(base_c + ((long long)p < rem ? 1 : 0));
          qmax = q[j] > qmax ? q[j] : qmax;
        }
        const int bits = qmax ? 64 - __clzll((long long)qmax) : 0;
        N.e = bits > 32 ? bits - 32 : 0;
        for (int j = 0; j < nb; ++j) N.m[j] = (unsigned)(q[j] >> N.e);
        tl.emitted += N.total(nb);
        tl.packets += 1;
        const float px = a.src_pos32[3 * s], py = a.src_pos32[3 * s + 1], pz = a.src_pos32[3 * s + 2];
        ix = a.src_cell[3 * s]; iy = a.src_cell[3 * s + 1]; iz = a.src_cell[3 * s + 2];
        // distances along the ray to the first x/y/z faces
        tMx = fx > 0.f ? ((float)(ix + 1) - px) / fx : (fx < 0.f ? ((float)ix - px) / fx : INFINITY);
        tMy = fy > 0.f ? ((float)(iy + 1) - py) / fy : (fy < 0.f ? ((float)iy - py) / fy : INFINITY);
        tMz = fz > 0.f ? ((float)(iz + 1) - pz) / fz : (fz < 0.f ? ((float)iz - pz) / fz : INFINITY);
        float trem = PER ? M->path_cells32 : 0.f;
        const int r = trace_mixed<NBT, HE, HEAT, PER>(ix, iy, iz, tMx, tMy, tMz, fx, fy, fz, N, M, a, t,
                                                      nb, S, tl, &trem);
        if (r == ESCAPED) tl.escaped += N.total(nb);
        alive = (r == ALIVE);
        // traced to the end (no queue to keep it): a packet still alive hit the DDA bound
        if (alive && S >= max_steps_all) atomicOr(a.err, ERR_DDA_LIMIT);
      }
    }
    if (S < max_steps_all)   // a wavefront launch: keep the survivors
      write_survivor<NBT>(a, w, alive, ix, iy, iz, b, tMx, tMy, tMz, fx, fy, fz, N, nb);
    flush_warp(a, b, tl);
  }
}

template <int NBT, bool HE, bool HEAT, int MINB, bool PER = false>
__global__ void __launch_bounds__(256, MINB) k_emit_mixed(StepArgs a, BinTables t, WFArgs w, int64_t g0,
                                                   int64_t n, int S, int max_steps_all) {
  emit_range<NBT, HE, HEAT, PER>(a, t, w, g0, n, S, max_steps_all);
}

// One re-emission packet per entry of this step's list (diffuse
// recombination field), traced to the end by its own thread: start point
// and direction from the cell's Philox counters, the photons of each species
// in its bin held as 32-bit counts of 2^e quanta as for a source packet.
// Entries are read in any order: deposits and counts do not depend on it.
template <int NBT, bool HE, bool HEAT, bool PER>
__global__ void __launch_bounds__(256, 3) k_rec_mixed(StepArgs a, BinTables t) {
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const int64_t n = (int64_t)*a.rec_count;
  const uint32_t step = (uint32_t)*a.step_dev;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = base + threadIdx.x;
    Tally tl{0, 0, 0, 0u, 0u};
    int b = -1;
    if (e < n) {
      const long long* L = a.rec_list + 4 * e;
      const int64_t g = L[0];
      b = box_of_cell(a.boxes, a.n_boxes, g);
      const BoxMeta* M = a.boxes + b;
      const int64_t cell = g - M->cell_off;
      float fx, fy, fz;
      if (!iso_direction_f32(M->seed, step, rec_src_id(cell), (uint32_t)cell, fx, fy, fz)) {
        atomicOr(a.err, ERR_DIRECTION);
      } else {
        unsigned long long q[NBT > 0 ? NBT : CRASH_MAX_BINS];
        for (int j = 0; j < nb; ++j) q[j] = 0ull;
        for (int s = 0; s < 3; ++s)
          if (a.rec_bin[s] >= 0) q[a.rec_bin[s]] += (unsigned long long)L[1 + s];
        unsigned long long qmax = 0;
        for (int j = 0; j < nb; ++j) qmax = q[j] > qmax ? q[j] : qmax;
        Content<NBT> N;
        const int bits = qmax ? 64 - __clzll((long long)qmax) : 0;
        N.e = bits > 32 ? bits - 32 : 0;
        for (int j = 0; j < nb; ++j) N.m[j] = (unsigned)(q[j] >> N.e);
        tl.emitted += N.total(nb);
        tl.packets += 1;
        double ox, oy, oz;
        rec_offsets(M->seed, step, cell, ox, oy, oz);
        int ix = (int)(cell % M->nx), iy = (int)((cell / M->nx) % M->ny);
        int iz = (int)(cell / ((int64_t)M->nx * M->ny));
        const float px = (float)((double)ix + ox), py = (float)((double)iy + oy);
        const float pz = (float)((double)iz + oz);
        float tMx = fx > 0.f ? ((float)(ix + 1) - px) / fx : (fx < 0.f ? ((float)ix - px) / fx : INFINITY);
        float tMy = fy > 0.f ? ((float)(iy + 1) - py) / fy : (fy < 0.f ? ((float)iy - py) / fy : INFINITY);
        float tMz = fz > 0.f ? ((float)(iz + 1) - pz) / fz : (fz < 0.f ? ((float)iz - pz) / fz : INFINITY);
        float trem = PER ? M->path_cells32 : 0.f;
        const int r = trace_mixed<NBT, HE, HEAT, PER>(ix, iy, iz, tMx, tMy, tMz, fx, fy, fz, N, M, a, t,
                                                      nb, M->max_iter, tl, &trem);
        if (r == ESCAPED) tl.escaped += N.total(nb);
        else if (r == ALIVE) atomicOr(a.err, ERR_DDA_LIMIT);
      }
    }
    flush_warp(a, b, tl);
  }
}

int num_sms();

template <int NBT, bool HE, bool HEAT>
void launch_rec_t(const StepArgs& a, const BinTables& t, cudaStream_t s) {
  if (a.any_periodic) k_rec_mixed<NBT, HE, HEAT, true><<<(unsigned)(num_sms() * 3), 256, 0, s>>>(a, t);
  else k_rec_mixed<NBT, HE, HEAT, false><<<(unsigned)(num_sms() * 3), 256, 0, s>>>(a, t);
}

// ------------------------------------------------------------------ passes
// One pass over the queue w.count_in holds, grid-stride over the calling
// grid: every packet advances at most S cells; survivors go to the output
// queue.  The queue is read through L2 (ld.global.cg): in the persistent
// launch other blocks of the same grid wrote it.
template <int NBT, bool HE, bool HEAT>
__device__ __forceinline__ void pass_range(const StepArgs& a, const BinTables& t, const WFArgs& w, int S) {
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const int64_t n = (int64_t)__ldcg(w.count_in);
  // the previous pass used the next pass's counter and has finished
  if (blockIdx.x == 0 && threadIdx.x == 0) *w.work_next = 0u;
  Tally tl{0, 0, 0, 0u, 0u};
  for (;;) {
    const int64_t base = next_block_packets(w.work);
    if (base >= n) break;
    const int64_t j = base + threadIdx.x;
    int b = -1;
    bool alive = false;
    int ix = 0, iy = 0, iz = 0;
    float tMx = 0.f, tMy = 0.f, tMz = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    Content<NBT> N;
    N.e = 0;
    if (j < n) {
      const int64_t i = w.perm ? (int64_t)__ldcg(w.perm + j) : j;
      load_record<NBT>(w.rec_in, w.rs, i, ix, iy, iz, b, tMx, tMy, tMz, fx, fy, fz, N, nb);
      const BoxMeta* M = a.boxes + b;
      const int r = trace_mixed<NBT, HE, HEAT>(ix, iy, iz, tMx, tMy, tMz, fx, fy, fz, N, M, a, t,
                                               nb, S, tl);
      if (r == ESCAPED) tl.escaped += N.total(nb);
      alive = (r == ALIVE);
    }
    write_survivor<NBT>(a, w, alive, ix, iy, iz, b, tMx, tMy, tMz, fx, fy, fz, N, nb);
    flush_warp(a, b, tl);
  }
}

template <int NBT, bool HE, bool HEAT, int MINB>
__global__ void __launch_bounds__(256, MINB) k_pass_mixed(StepArgs a, BinTables t, WFArgs w, int S) {
  pass_range<NBT, HE, HEAT>(a, t, w, S);
}

// The same pass for the persistent launch, the input queue CUR (0 or 1)
// fixed at compile time: its pointers are read from the kernel's parameter
// bank as in the one-launch-per-pass kernel instead of occupying registers.
template <int NBT, bool HE, bool HEAT, int CUR>
__device__ __forceinline__ void pass_range_q(const StepArgs& a, const BinTables& t, const WF& wf, int S,
                                             bool read_sorted, bool write_keys, int curve) {
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const int64_t n = (int64_t)__ldcg(wf.count + CUR);
  Tally tl{0, 0, 0, 0u, 0u};
  for (;;) {
    const int64_t base = next_block_packets(wf.count + 2);   // cleared before the pass
    if (base >= n) break;
    const int64_t j = base + threadIdx.x;
    int b = -1;
    bool alive = false;
    int ix = 0, iy = 0, iz = 0;
    float tMx = 0.f, tMy = 0.f, tMz = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    Content<NBT> N;
    N.e = 0;
    if (j < n) {
      const int64_t i = read_sorted ? (int64_t)__ldcg(wf.perm + j) : j;
      load_record<NBT>(wf.rec[CUR], wf.rs, i, ix, iy, iz, b, tMx, tMy, tMz, fx, fy, fz, N, nb);
      const BoxMeta* M = a.boxes + b;
      const int r = trace_mixed<NBT, HE, HEAT>(ix, iy, iz, tMx, tMy, tMz, fx, fy, fz, N, M, a, t,
                                               nb, S, tl);
      if (r == ESCAPED) tl.escaped += N.total(nb);
      alive = (r == ALIVE);
    }
    write_survivor_to<NBT>(a, wf.count + (1 - CUR), wf.cap, wf.rec[1 - CUR], wf.rs, write_keys, wf.key, wf.rank,
                           wf.bcount, 0, curve, alive, ix, iy, iz, b, tMx, tMy, tMz, fx, fy, fz, N, nb);
    flush_warp(a, b, tl);
  }
}

// ------------------------------------------------------------------ re-sort
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

// sorted position of record j: boff[key] + rank
__global__ void k_perm(const unsigned* count, const unsigned* key, const unsigned* rank,
                       const unsigned* boff, unsigned* perm, int* err) {
  const int64_t n = (int64_t)*count;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const int64_t d = (int64_t)boff[key[j]] + rank[j];
    if (d >= n) { atomicOr(err, ERR_QUEUE); continue; }
    perm[d] = (unsigned)j;
  }
}

// ------------------------------------------------------------------ tiles
constexpr int kTileItem = 8192;        // packets of a tile handled by one block visit
constexpr int kTileBlock = 768;        // one block per SM (shared memory)
constexpr size_t kTileSmem = 4096 * sizeof(float4) + 4096 * 4 * sizeof(unsigned long long);

__device__ __forceinline__ unsigned compact3(unsigned v) {   // every third bit -> 10 bits
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030C30C3u;
  v = (v | (v >> 4)) & 0x0300F00Fu;
  v = (v | (v >> 8)) & 0x030000FFu;
  v = (v | (v >> 16)) & 0x3FFu;
  return v;
}

__device__ __forceinline__ int box_of_tile(const BoxMeta* b, int n, unsigned T) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((unsigned)(b[mid].tile_off >> 3) <= T) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// packets of tile T occupy sorted positions [boff[8T], boff[8T+8])
__device__ __forceinline__ unsigned tile_end(const unsigned* boff, const unsigned* count, int64_t n_keys,
                                             unsigned T) {
  return (8 * (int64_t)T + 8 < n_keys) ? boff[8 * (int64_t)T + 8] : *count;
}

// work items of a tile pass: (tile, first sorted position), at most
// kTileItem packets each, in any order (results do not depend on it)
__global__ void k_tile_list(const unsigned* boff, const unsigned* count, int64_t n_keys, uint2* items,
                            unsigned* nitems) {
  const int64_t ntiles = n_keys / 8;
  for (int64_t T = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; T < ntiles;
       T += (int64_t)gridDim.x * blockDim.x) {
    const unsigned lo = boff[8 * T], hi = tile_end(boff, count, n_keys, (unsigned)T);
    if (hi > lo) {
      const unsigned k = (hi - lo + kTileItem - 1) / kTileItem;
      const unsigned at = atomicAdd(nitems, k);
      for (unsigned q = 0; q < k; ++q) items[at + q] = make_uint2((unsigned)T, lo + q * kTileItem);
    }
  }
}

// One tile pass: a block takes the next work item (up to kTileItem packets
// of one 16^3 tile), stages the tile's absorbers in shared memory with its
// deposits zeroed, and its warps take the item's packets 32 at a time and
// walk each until it leaves the tile (or is absorbed or escapes).  Deposits
// are int64 atomics in shared memory; once the item is done every cell that
// received any adds it to the grid with one reduction per species, so the
// grid's deposit array is touched once per item instead of once per
// crossing.  Sums of integers do not depend on their order: the deposits
// are the same bits as with per-crossing reductions.  Survivors go to the
// output queue with the key of the tile they enter.
template <int NBT, bool HE, bool HEAT>
__global__ void __launch_bounds__(kTileBlock, 1) k_tile_pass(StepArgs a, BinTables t, WFArgs w,
                                                             const unsigned* boff, const uint2* items,
                                                             const unsigned* nitems, unsigned* next,
                                                             int64_t n_keys) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sabs = reinterpret_cast<float4*>(smem);
  unsigned long long* sdep = reinterpret_cast<unsigned long long*>(smem + 4096 * sizeof(float4));
  __shared__ unsigned s_item, s_next;
  const unsigned full = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const int nb = NBT > 0 ? NBT : t.n_bins;
  const unsigned nit = *nitems;
  const float4* abs32 = reinterpret_cast<const float4*>(a.abs32);
  Tally tl{0, 0, 0, 0u, 0u};
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1u);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= nit) break;
    const uint2 it = items[item];
    const unsigned T = it.x;
    const int b = box_of_tile(a.boxes, a.n_boxes, T);
    const BoxMeta* M = a.boxes + b;
    const unsigned lt = T - (unsigned)(M->tile_off >> 3);
    const int x0 = 16 * (int)compact3(lt), y0 = 16 * (int)compact3(lt >> 1), z0 = 16 * (int)compact3(lt >> 2);
    const int ex = min(16, M->nx - x0), ey = min(16, M->ny - y0), ez = min(16, M->nz - z0);
    const unsigned lo = it.y;
    const unsigned hi = min(lo + (unsigned)kTileItem, tile_end(boff, w.count_in, n_keys, T));
    for (int li = threadIdx.x; li < 4096; li += blockDim.x) {
      const int lx = li & 15, ly = (li >> 4) & 15, lz = li >> 8;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (lx < ex && ly < ey && lz < ez)
        v = __ldg(abs32 + M->cell_off + (x0 + lx) + M->nx * ((y0 + ly) + M->ny * (z0 + lz)));
      sabs[li] = v;
      sdep[li] = 0ull;
      sdep[4096 + li] = 0ull;
      sdep[8192 + li] = 0ull;
      sdep[12288 + li] = 0ull;
    }
    if (threadIdx.x == 0) s_next = lo;
    __syncthreads();
    const TileCells cells{sabs, sdep, x0, y0, z0};
    for (;;) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(&s_next, 32u);
      base = __shfl_sync(full, base, 0);
      if (base >= hi) break;
      const unsigned j = base + lane;
      int pb = -1;
      bool alive = false;
      int ix = 0, iy = 0, iz = 0;
      float tMx = 0.f, tMy = 0.f, tMz = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
      Content<NBT> N;
      N.e = 0;
      if (j < hi) {
        load_record<NBT>(w.rec_in, w.rs, (long long)w.perm[j], ix, iy, iz, pb, tMx, tMy, tMz, fx, fy, fz,
                         N, nb);
        const int r = walk<NBT, HE, HEAT, true, false>(ix, iy, iz, tMx, tMy, tMz, fx, fy, fz, N, M, cells,
                                                       t, nb, 64, tl, x0, y0, z0, ex, ey, ez);
        if (r == ESCAPED) tl.escaped += N.total(nb);
        alive = (r == ALIVE);
      }
      write_survivor<NBT>(a, w, alive, ix, iy, iz, pb, tMx, tMy, tMz, fx, fy, fz, N, nb);
      flush_warp(a, pb, tl);
    }
    __syncthreads();
    // the item's deposits to the grid, cell by cell
    for (int li = threadIdx.x; li < 4096; li += blockDim.x) {
      const int lx = li & 15, ly = (li >> 4) & 15, lz = li >> 8;
      if (lx < ex && ly < ey && lz < ez) {
        unsigned long long* g = a.dep + 4 * (M->cell_off + (x0 + lx) + (int64_t)M->nx * ((y0 + ly) + (int64_t)M->ny * (z0 + lz)));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const unsigned long long v = sdep[4096 * k + li];
          if (v) atomicAdd(g + k, v);
        }
      }
    }
    __syncthreads();
  }
}

__global__ void k_check_drained(const unsigned* count, int* err) {
  if (*count != 0u) atomicOr(err, ERR_WATCHDOG);
}

__host__ __device__ __forceinline__ WFArgs wf_args(const WF& wf, int in, bool read_sorted, bool write_keys,
                                                    int tile = 0, int curve = 0) {
  WFArgs w;
  w.tile = tile;
  w.curve = curve;
  const int out = 1 - in;
  w.rec_in = wf.rec[in];
  w.rec_out = wf.rec[out];
  w.count_in = wf.count + in;
  w.count_out = wf.count + out;
  w.perm = read_sorted ? wf.perm : nullptr;
  w.key = write_keys ? wf.key : nullptr;
  w.rank = write_keys ? wf.rank : nullptr;
  w.bcount = wf.bcount;
  w.rs = wf.rs;
  w.cap = wf.cap;
  w.work = nullptr;
  w.work_next = nullptr;
  return w;
}
WFArgs wf_args(WF* wf, int in, bool read_sorted, bool write_keys, int tile = 0, int curve = 0) {
  return wf_args(*wf, in, read_sorted, write_keys, tile, curve);
}

// ------------------------------------------------------------------ persistent
// Grid barrier of a cooperative launch (every block resident at once): a
// block arrives, then waits until the last one to arrive advances the
// generation word.  Every wait is bounded by kBarrierLimitNs of %globaltimer
// and ends early once any block has set the error word; false means the
// launch stops (the host then reports the error word).
constexpr unsigned long long kBarrierLimitNs = 30ull * 1000000000ull;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_sync(unsigned* gs, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire_u32(gs + 1);      // read before arriving
    __threadfence();                                  // this block's writes, device-wide
    if (atomicAdd(gs, 1u) == gridDim.x - 1) {
      atomicExch(gs, 0u);
      __threadfence();
      atomicAdd(gs + 1, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (ld_acquire_u32(gs + 1) == gen) {
        if (*(volatile int*)err != 0) { ok = 0; break; }
        if (globaltimer_ns() - t0 > kBarrierLimitNs) {
          atomicOr(err, ERR_WATCHDOG);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = ok && *(volatile int*)err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// The whole wavefront transport of a step in one cooperative launch: chunk
// after chunk of at most wf.cap packets, emission into queue 0, then the
// passes, each reading the queue the previous one wrote; before a sorted pass
// the counting sort runs in three phases between grid barriers (segment
// scans of the key counts, the scan of the segment sums, the sorted position
// boff[key] + bsum[key / 4096] + rank of every record).  The same device code
// as the one-launch-per-pass sequence, so the deposits are the same bits.
template <int NBT, bool HE, bool HEAT, int MINB>
__global__ void __launch_bounds__(256, MINB) k_wavefront(StepArgs a, BinTables t, WF wf, int S, int R,
                                                         int passes, int curve, int max_iter) {
  __shared__ unsigned sh[32];
  // the loop state lives in shared memory so that it holds no registers
  // across the passes (the pass body needs every register of the cap)
  __shared__ volatile long long s_g0;
  __shared__ volatile int s_p, s_cur;
  auto sorted_pass = [&](int p) { return p >= 1 && p < passes && R > 0 && (p % R) == 0; };
  if (threadIdx.x == 0) s_g0 = 0;
  __syncthreads();
  while (s_g0 < a.total_packets) {
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g0 = s_g0;
    const int64_t n = a.total_packets - g0 < wf.cap ? a.total_packets - g0 : wf.cap;
    if (gtid == 0) {
      wf.count[0] = 0u;
      wf.count[1] = 0u;
    }
    if (sorted_pass(1))
      for (int64_t k = gtid; k < wf.n_keys; k += gstride) wf.bcount[k] = 0u;
    if (!grid_sync(wf.gsync, a.err)) return;
    emit_range<NBT, HE, HEAT, false>(a, t, wf_args(wf, 1, false, sorted_pass(1), 0, curve), g0, n, 0,
                                     max_iter);
    if (!grid_sync(wf.gsync, a.err)) return;
    if (threadIdx.x == 0) {
      s_p = 1;
      s_cur = 0;
    }
    __syncthreads();
    while (s_p < passes) {
      const int p = s_p, cur = s_cur;
      const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
      const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
      const bool sorted_now = sorted_pass(p), keys_next = sorted_pass(p + 1);
      if (sorted_now) {
        const int64_t nk = wf.n_keys;
        const int64_t nseg = (nk + 4095) / 4096;
        for (int64_t seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
          const int64_t base = seg * 4096 + (int64_t)threadIdx.x * 16;
          unsigned v[16], sum = 0u;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            v[k] = base + k < nk ? __ldcg(wf.bcount + base + k) : 0u;
            sum += v[k];
          }
          unsigned tot;
          unsigned ex = block_excl_scan(sum, sh, &tot);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            if (base + k < nk) wf.boff[base + k] = ex;
            ex += v[k];
          }
          if (threadIdx.x == 0) wf.bsum[seg] = tot;
        }
        if (!grid_sync(wf.gsync, a.err)) return;
        if (blockIdx.x == 0) {
          unsigned v[4], sum = 0u;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int64_t idx = (int64_t)threadIdx.x * 4 + k;
            v[k] = idx < nseg ? __ldcg(wf.bsum + idx) : 0u;
            sum += v[k];
          }
          unsigned tot;
          unsigned ex = block_excl_scan(sum, sh, &tot);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int64_t idx = (int64_t)threadIdx.x * 4 + k;
            if (idx < nseg) wf.bsum[idx] = ex;
            ex += v[k];
          }
        }
        if (!grid_sync(wf.gsync, a.err)) return;
        const int64_t cnt = (int64_t)__ldcg(wf.count + cur);
        for (int64_t j = gtid; j < cnt; j += gstride) {
          const unsigned k = __ldcg(wf.key + j);
          const int64_t d = (int64_t)__ldcg(wf.boff + k) + __ldcg(wf.bsum + (k >> 12)) + __ldcg(wf.rank + j);
          if (d >= cnt) atomicOr(a.err, ERR_QUEUE);
          else wf.perm[d] = (unsigned)j;
        }
      }
      if (keys_next)
        for (int64_t k = gtid; k < wf.n_keys; k += gstride) wf.bcount[k] = 0u;
      if (gtid == 0) {
        wf.count[1 - cur] = 0u;
        wf.count[2] = 0u;          // the pass's work counter
      }
      if (!grid_sync(wf.gsync, a.err)) return;
      if (cur == 0) pass_range_q<NBT, HE, HEAT, 0>(a, t, wf, S, sorted_now, keys_next, curve);
      else pass_range_q<NBT, HE, HEAT, 1>(a, t, wf, S, sorted_now, keys_next, curve);
      if (!grid_sync(wf.gsync, a.err)) return;
      if (threadIdx.x == 0) {
        s_cur = 1 - s_cur;
        s_p = s_p + 1;
      }
      __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && __ldcg(wf.count + s_cur) != 0u) atomicOr(a.err, ERR_WATCHDOG);
    if (!grid_sync(wf.gsync, a.err)) return;
    if (threadIdx.x == 0) s_g0 = s_g0 + wf.cap;
    __syncthreads();
  }
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
  if (a.any_periodic) {
    // periodic boxes: one thread per packet, traced to the end of its c dt
    int64_t blocks = (a.total_packets + block - 1) / block;
    if (blocks > (int64_t)1 << 30) blocks = (int64_t)1 << 30;
    WFArgs w = wf_args(wf, 0, false, false);
    tic();
    k_emit_mixed<NBT, HE, HEAT, 3, true><<<(unsigned)blocks, block, 0, s>>>(a, t, w, 0, a.total_packets,
                                                                         max_iter, max_iter);
    toc();
    return 1;
  }
  if (!o.wavefront || wf->cap == 0) {
    // one thread per packet, traced to the end
    WFArgs w = wf_args(wf, 0, false, false);
    int64_t blocks = (a.total_packets + block - 1) / block;
    if (blocks > (int64_t)1 << 30) blocks = (int64_t)1 << 30;
    tic();
    if (o.reg_cap)
      k_emit_mixed<NBT, HE, HEAT, 4><<<(unsigned)blocks, block, 0, s>>>(a, t, w, 0, a.total_packets,
                                                                       max_iter, max_iter);
    else
      k_emit_mixed<NBT, HE, HEAT, 3><<<(unsigned)blocks, block, 0, s>>>(a, t, w, 0, a.total_packets,
                                                                       max_iter, max_iter);
    toc();
    return 1;
  }
  if (o.tile && wf->items) {
    // emission only (no walk), then tile passes until every packet is done
    static bool smem_set = false;
    if (!smem_set) {
      cudaFuncSetAttribute(k_tile_pass<NBT, HE, HEAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTileSmem);
      smem_set = true;
    }
    const int64_t nk = a.n_tile_keys;
    const int nscan_t = (int)((nk + 4095) / 4096);
    for (int64_t g0 = 0; g0 < a.total_packets; g0 += wf->cap) {
      const int64_t n = std::min<int64_t>(wf->cap, a.total_packets - g0);
      int cur = 1;
      cudaMemsetAsync(wf->count, 0, 4 * sizeof(unsigned), s);
      cudaMemsetAsync(wf->bcount, 0, sizeof(unsigned) * nk, s);
      {
        WFArgs w = wf_args(wf, cur, false, true, 1, o.sort_curve);
        int64_t blocks = (n + block - 1) / block;
        if (blocks > persistent * 4) blocks = persistent * 4;
        tic();
        k_emit_mixed<NBT, HE, HEAT, 3><<<(unsigned)blocks, block, 0, s>>>(a, t, w, g0, n, 0, max_iter);
        toc();
        ++launches;
        cur = 0;
      }
      const int tile_passes = (o.pass_limit > 0 && o.pass_limit < a.max_tiles) ? o.pass_limit : a.max_tiles;
      for (int p = 1; p <= tile_passes; ++p) {
        k_scan_blocks<<<nscan_t, 1024, 0, s>>>(wf->bcount, wf->boff, wf->bsum, nk);
        k_scan_sums<<<1, 1024, 0, s>>>(wf->bsum, nscan_t);
        k_scan_add<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(wf->boff, wf->bsum, nk);
        k_perm<<<persistent, block, 0, s>>>(wf->count + cur, wf->key, wf->rank, wf->boff, wf->perm, a.err);
        cudaMemsetAsync(wf->count + 2, 0, 2 * sizeof(unsigned), s);
        k_tile_list<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((nk / 8 + 255) / 256, 4096)), 256, 0, s>>>(
            wf->boff, wf->count + cur, nk, wf->items, wf->count + 2);
        cudaMemsetAsync(wf->bcount, 0, sizeof(unsigned) * nk, s);
        WFArgs w = wf_args(wf, cur, true, true, 1, o.sort_curve);
        cudaMemsetAsync(w.count_out, 0, sizeof(unsigned), s);
        tic();
        k_tile_pass<NBT, HE, HEAT><<<num_sms(), kTileBlock, kTileSmem, s>>>(
            a, t, w, wf->boff, wf->items, wf->count + 2, wf->count + 3, nk);
        toc();
        launches += 6;
        cur = 1 - cur;
      }
      k_check_drained<<<1, 1, 0, s>>>(wf->count + cur, a.err);
      ++launches;
    }
    return launches;
  }
  const int S = o.seg_per_iter > 0 ? o.seg_per_iter : 32;
  const int R = o.resort_interval == 0 ? 1 : o.resort_interval;
  // emission only writes the packets (no walk): every crossing is made by the
  // passes, which read the queue in sorted order
  int passes = (max_iter + S - 1) / S + 1;
  if (o.pass_limit > 0 && o.pass_limit < passes) passes = o.pass_limit;
  if (o.persistent && wf->gsync) {
    // one cooperative launch for the whole step (all blocks resident)
    static int per_sm[2] = {0, 0};
    const int ci = o.reg_cap ? 1 : 0;
    if (!per_sm[ci]) {
      if (o.reg_cap)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[ci], k_wavefront<NBT, HE, HEAT, 4>, 256, 0);
      else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[ci], k_wavefront<NBT, HE, HEAT, 3>, 256, 0);
    }
    if (per_sm[ci] < 1) return -1;
    cudaMemsetAsync(wf->gsync, 0, 2 * sizeof(unsigned), s);
    WF wv = *wf;
    StepArgs av = a;
    BinTables tv = t;
    int Sv = S, Rv = R, pv = passes, cv = o.sort_curve, mv = max_iter;
    void* args[] = {&av, &tv, &wv, &Sv, &Rv, &pv, &cv, &mv};
    tic();
    const cudaError_t e = o.reg_cap
        ? cudaLaunchCooperativeKernel((const void*)k_wavefront<NBT, HE, HEAT, 4>, num_sms() * per_sm[ci], 256, args, 0, s)
        : cudaLaunchCooperativeKernel((const void*)k_wavefront<NBT, HE, HEAT, 3>, num_sms() * per_sm[ci], 256, args, 0, s);
    toc();
    return e == cudaSuccess ? 1 : -1;
  }
  const int nscan = (int)((wf->n_keys + 4095) / 4096);
  // the pass p (p >= 1) reads in sorted order when R > 0 and p % R == 0
  auto sorted_pass = [&](int p) { return p >= 1 && p < passes && R > 0 && (p % R) == 0; };
  for (int64_t g0 = 0; g0 < a.total_packets; g0 += wf->cap) {
    const int64_t n = std::min<int64_t>(wf->cap, a.total_packets - g0);
    int cur = 1;   // emission reads nothing and writes buffer 0
    cudaMemsetAsync(wf->count, 0, 4 * sizeof(unsigned), s);
    for (int p = 0; p < passes; ++p) {
      const bool next_sorted = sorted_pass(p + 1);
      if (next_sorted) cudaMemsetAsync(wf->bcount, 0, sizeof(unsigned) * wf->n_keys, s);
      WFArgs w = wf_args(wf, cur, sorted_pass(p), next_sorted, 0, o.sort_curve);
      // pass p hands out its queue from count[2 + p % 2] and clears the
      // other one for pass p + 1 (both are cleared with the chunk)
      w.work = wf->count + 2 + (p & 1);
      w.work_next = wf->count + 2 + ((p + 1) & 1);
      cudaMemsetAsync(w.count_out, 0, sizeof(unsigned), s);
      tic();
      if (p == 0) {
        int64_t blocks = (n + block - 1) / block;
        if (blocks > persistent * 4) blocks = persistent * 4;
        if (o.reg_cap)
          k_emit_mixed<NBT, HE, HEAT, 4><<<(unsigned)blocks, block, 0, s>>>(a, t, w, g0, n, 0, max_iter);
        else
          k_emit_mixed<NBT, HE, HEAT, 3><<<(unsigned)blocks, block, 0, s>>>(a, t, w, g0, n, 0, max_iter);
      } else {
        if (o.reg_cap) k_pass_mixed<NBT, HE, HEAT, 4><<<persistent, block, 0, s>>>(a, t, w, S);
        else k_pass_mixed<NBT, HE, HEAT, 3><<<persistent, block, 0, s>>>(a, t, w, S);
      }
      toc();
      ++launches;
      cur = 1 - cur;
      if (next_sorted) {
        k_scan_blocks<<<nscan, 1024, 0, s>>>(wf->bcount, wf->boff, wf->bsum, wf->n_keys);
        k_scan_sums<<<1, 1024, 0, s>>>(wf->bsum, nscan);
        k_scan_add<<<(unsigned)((wf->n_keys + 255) / 256), 256, 0, s>>>(wf->boff, wf->bsum, wf->n_keys);
        k_perm<<<persistent, block, 0, s>>>(wf->count + cur, wf->key, wf->rank, wf->boff, wf->perm, a.err);
        launches += 4;
      }
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

int launch_trace_mixed_external(const StepArgs& a, const BinTables& t, const crash_run_opts& o,
                                char* rec0, char* rec1, unsigned* count, int64_t cap, int max_iter,
                                cudaStream_t s) {
  WF wf;                       // views the caller's buffers; owns nothing
  wf.cap = cap;
  wf.nb = t.n_bins;
  wf.rs = ((32 + 4 * t.n_bins) + 15) / 16 * 16;
  wf.rec[0] = rec0;
  wf.rec[1] = rec1;
  wf.count = count;
  crash_run_opts oo = o;
  oo.wavefront = 1;
  oo.resort_interval = -1;     // no sort keys without their workspace
  oo.tile = 0;
  oo.persistent = 0;           // no grid barrier word either
  return launch_trace_mixed(a, t, oo, &wf, max_iter, s, nullptr, nullptr);
}

void* wavefront_create(int64_t cap, int64_t n_keys, int nb, cudaError_t* err) {
  WF* w = new WF();
  w->cap = cap;
  w->nb = nb;
  w->rs = ((32 + 4 * nb) + 15) / 16 * 16;
  w->n_keys = n_keys;
  cudaError_t e = cudaMalloc(&w->count, 4 * sizeof(unsigned));
  if (e == cudaSuccess && cap > 0) {
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&w->rec[b], (size_t)w->rs * cap);
    if (e == cudaSuccess) e = cudaMalloc(&w->key, sizeof(unsigned) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&w->rank, sizeof(unsigned) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&w->perm, sizeof(unsigned) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&w->bcount, sizeof(unsigned) * n_keys);
    if (e == cudaSuccess) e = cudaMalloc(&w->boff, sizeof(unsigned) * n_keys);
    if (e == cudaSuccess) e = cudaMalloc(&w->bsum, sizeof(unsigned) * 1024);
    if (e == cudaSuccess) e = cudaMalloc(&w->items, sizeof(uint2) * (n_keys / 8 + cap / 2048 + 2));
    if (e == cudaSuccess) e = cudaMalloc(&w->gsync, 2 * sizeof(unsigned));
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
  void* ptrs[] = {w->count, w->key, w->rank, w->perm, w->bcount, w->boff, w->bsum, w->items,
                  w->gsync, w->rec[0], w->rec[1]};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete w;
}

int64_t wavefront_capacity(void* p) { return p ? ((WF*)p)->cap : 0; }

int launch_rec_mixed(const StepArgs& a, const BinTables& t, cudaStream_t s) {
  const bool he = a.any_he != 0, heat = a.any_heat != 0;
  if (t.n_bins == 1) {
    if (he) { if (heat) launch_rec_t<1, true, true>(a, t, s); else launch_rec_t<1, true, false>(a, t, s); }
    else { if (heat) launch_rec_t<1, false, true>(a, t, s); else launch_rec_t<1, false, false>(a, t, s); }
  } else if (t.n_bins == 8) {
    if (he) { if (heat) launch_rec_t<8, true, true>(a, t, s); else launch_rec_t<8, true, false>(a, t, s); }
    else { if (heat) launch_rec_t<8, false, true>(a, t, s); else launch_rec_t<8, false, false>(a, t, s); }
  } else {
    if (he) { if (heat) launch_rec_t<0, true, true>(a, t, s); else launch_rec_t<0, true, false>(a, t, s); }
    else { if (heat) launch_rec_t<0, false, true>(a, t, s); else launch_rec_t<0, false, false>(a, t, s); }
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}
