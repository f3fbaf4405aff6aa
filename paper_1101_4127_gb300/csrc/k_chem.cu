// k_chem.cu -- per-cell ionisation network and temperature update (FP64),
// one thread per cell over all boxes, reading the step's integer deposits.
//
// Sec. 2: each cell's ionisation fractions change by photo-ionisation (the
// absorbed photons), collisional ionisation and recombination, and its
// temperature by photo-heating, the change in the number of free particles
// and the continuous processes (bremsstrahlung, Compton, collisional
// ionisation and excitation cooling, recombination cooling).  Sec. 3.2: the
// network is sub-sampled when the step exceeds its time-scales.
//
// Coupling of transport to chemistry (step-synchronous form): the step's
// deposit of species s, dep_s quanta of 2^E photons, defines either
//   * (coupling 0) a photo-ionisation rate per absorber
//     Gamma_s = dep_s 2^E / (dt n_s^0 V) with n_s^0 the absorber density
//     frozen at the start of the step; photo-heating is the mean excess
//     energy per absorbed photon times the photo-ionisation rate of the
//     current absorbers; or
//   * (coupling 1, photon-conserving) a constant source of dep_s 2^E / (dt V)
//     ionisations per cm^3 and s, in each sub-step at most the atoms of the
//     species present (the photons beyond are lost); photo-heating at the
//     constant deposited rate.
//
// Integrator per sub-step h (h limited so that no ionic fraction changes by
// more than eps * max(x, 1e-3) and T by more than eps * T; the last allowed
// sub-step takes what remains):
//   * backward Euler for the H (2-state) and He (3-state tridiagonal) chains
//     at fixed T, with n_e at the end of the sub-step by at most 4
//     fixed-point passes (fewer once n_e changes by less than 1e-12);
//   * fractions clamped to [0,1], He renormalised to unit sum;
//   * 1.5 k (n_tot T)_new = 1.5 k (n_tot T)_old + h (H + C n_e T_cmb)
//     - h (Lambda(T_old)/T_old + C n_e) T_new  (cooling linear in T_new).
// With the diffuse recombination field on (f_rec > 0) the network uses case
// A and counts the recombinations straight to the ground state of each ion,
// which the next step re-emits as packets.
#include <math.h>

#include <algorithm>

#include "crash_internal.cuh"
#include "k_device.cuh"

using namespace crash;

namespace {

constexpr double kB = 1.380649e-16;
constexpr double eV = 1.602176634e-12;
constexpr double sigmaT = 6.6524587321e-25;
constexpr double aRad = 7.565723e-15;
constexpr double mE = 9.1093837015e-28;
constexpr double cLight = 2.99792458e10;

struct Rates {
  double aHII, aHeII, aHeIII, adiel;     // recombination, cm^3/s
  double bHI, bHeI, bHeII;               // collisional ionisation, cm^3/s
  double cexHI, cexHeII;                 // collisional excitation cooling, erg cm^3/s
  double cionHI, cionHeI, cionHeII;      // collisional ionisation cooling
  double crecHII, crecHeII, crecHeIII;   // recombination cooling
  double cdiel;                          // dielectronic recombination cooling
  double cff;                            // bremsstrahlung per Z^2 (times n_e n_i)
};

// Hui & Gnedin (1997) recombination (case A/B) and recombination cooling;
// Cen (1992) collisional ionisation, collisional excitation cooling and
// dielectronic recombination; bremsstrahlung 1.42e-27 g_ff sqrt(T).
// R = double in the FP64 form; R = float in the mixed form, where the fits
// (themselves accurate to a few per cent) are evaluated in FP32 and the
// integration stays in FP64.
template <typename R>
__device__ Rates rates_at(double Td, int caseB) {
  Rates r;
  const R T = (R)Td;
  const R one = (R)1, lH = (R)315614.0 / T, lHe1 = (R)570670.0 / T, lHe2 = (R)1263030.0 / T;
  const R sq = one / (one + sqrt(T / (R)1e5));
  if (caseB) {
    r.aHII = (R)2.753e-14 * pow(lH, (R)1.5) / pow(one + pow(lH / (R)2.740, (R)0.407), (R)2.242);
    r.aHeII = (R)1.26e-14 * pow(lHe1, (R)0.750);
    r.aHeIII = (R)2 * (R)2.753e-14 * pow(lHe2, (R)1.5) / pow(one + pow(lHe2 / (R)2.740, (R)0.407), (R)2.242);
    r.crecHII = (double)((R)3.435e-30 * T * pow(lH, (R)1.970) / pow(one + pow(lH / (R)2.250, (R)0.376), (R)3.720));
    r.crecHeIII = (double)((R)8 * (R)3.435e-30 * ((R)0.25 * T) * pow(lHe2, (R)1.970) /
                           pow(one + pow(lHe2 / (R)2.250, (R)0.376), (R)3.720));
  } else {
    r.aHII = (R)1.269e-13 * pow(lH, (R)1.503) / pow(one + pow(lH / (R)0.522, (R)0.470), (R)1.923);
    r.aHeII = (R)3.0e-14 * pow(lHe1, (R)0.654);
    r.aHeIII = (R)2 * (R)1.269e-13 * pow(lHe2, (R)1.503) / pow(one + pow(lHe2 / (R)0.522, (R)0.470), (R)1.923);
    r.crecHII = (double)((R)1.778e-29 * T * pow(lH, (R)1.965) / pow(one + pow(lH / (R)0.541, (R)0.502), (R)2.697));
    r.crecHeIII = (double)((R)8 * (R)1.778e-29 * ((R)0.25 * T) * pow(lHe2, (R)1.965) /
                           pow(one + pow(lHe2 / (R)0.541, (R)0.502), (R)2.697));
  }
  r.adiel = (double)((R)1.90e-3 * pow(T, (R)-1.5) * exp((R)-470000.0 / T) * (one + (R)0.3 * exp((R)-94000.0 / T)));
  const R rt = sqrt(T);
  const R bHI = (R)5.85e-11 * rt * exp((R)-157809.1 / T) * sq;
  const R bHeI = (R)2.38e-11 * rt * exp((R)-285335.4 / T) * sq;
  const R bHeII = (R)5.68e-12 * rt * exp((R)-631515.0 / T) * sq;
  r.bHI = bHI; r.bHeI = bHeI; r.bHeII = bHeII;
  const R lg = log10(T);
  const R gff = (R)1.1 + (R)0.34 * exp(-((R)5.5 - lg) * ((R)5.5 - lg) / (R)3.0);
  r.cexHI = (double)((R)7.50e-19 * exp((R)-118348.0 / T) * sq);
  r.cexHeII = (double)((R)5.54e-17 * pow(T, (R)-0.397) * exp((R)-473638.0 / T) * sq);
  r.cionHI = 13.6 * eV * r.bHI;
  r.cionHeI = 24.6 * eV * r.bHeI;
  r.cionHeII = 54.4 * eV * r.bHeII;
  r.crecHeII = kB * Td * r.aHeII;
  r.cdiel = 6.526e-11 * r.adiel;
  r.cff = (double)((R)1.42e-27 * gff * rt);
  return r;
}

__device__ __forceinline__ double cooling_rate(const Rates& r, int mask, double ne, double nHI,
                                               double nHII, double nHeI, double nHeII,
                                               double nHeIII) {
  double L = 0.0;
  if (mask & 1) L += ne * (r.cexHI * nHI + r.cexHeII * nHeII);
  if (mask & 2) L += ne * (r.cionHI * nHI + r.cionHeI * nHeI + r.cionHeII * nHeII);
  if (mask & 4) L += ne * (r.crecHII * nHII + r.crecHeII * nHeII + r.crecHeIII * nHeIII);
  if (mask & 32) L += ne * r.cdiel * nHeII;
  if (mask & 8) L += ne * r.cff * (nHII + nHeII + 4.0 * nHeIII);
  return L;
}

struct CellIn {
  // GH, G1, G2: photo-ionisation rate per absorber, from the deposits plus
  // the uniform background; WH, W1, W2: photo-heating per absorber (erg/s),
  // the deposits' mean excess energy times their rate plus the background's
  // heat per ionisation times its rate
  double nH, nHe, GH, G1, G2, WH, W1, W2, Tcmb, ccomp, eps, V;
  double SH, S1, S2, heat_rate;   // constant sources per atom of the element (s^-1), erg/cm^3/s
  int iso, caseB, mask, max_sub, count_rec;
};

// One sub-step of the cell integration; updates x (HII), y2 (HeII), y3
// (HeIII), T and the remaining time rem (0 after the last sub-step).  COUNT
// (diffuse recombination field): adds to nrec[] the recombinations straight
// to the ground state of H I, He I, He II per cm^3 in the sub-step,
// (alpha_A - alpha_B) n_e n_ion (at least 0) with the rates at the
// sub-step's starting temperature and n_e and the ions at its end, as in
// the backward-Euler update.
template <typename RT, bool COUNT>
__device__ __forceinline__ void substep(const CellIn& c, double& x, double& y2, double& y3, double& T,
                                        double& rem, int nsub, double* nrec) {
  const bool coll = (c.mask & 2) != 0, rec = (c.mask & 4) != 0, diel = (c.mask & 32) != 0;
  const bool he = c.nHe > 0.0;
  const Rates r = rates_at<RT>(T, c.caseB);
  double gH = 0.0, g2 = 0.0, g3 = 0.0;
  if (COUNT && c.count_rec && rec) {
    const Rates rB = rates_at<RT>(T, 1);
    gH = fmax(r.aHII - rB.aHII, 0.0);
    g2 = fmax(r.aHeII - rB.aHeII, 0.0);
    g3 = fmax(r.aHeIII - rB.aHeIII, 0.0);
  }
  const double aH = rec ? r.aHII : 0.0;
  const double aHe2 = rec ? r.aHeII + (diel ? r.adiel : 0.0) : 0.0;
  const double aHe3 = rec ? r.aHeIII : 0.0;
  const double bH = coll ? r.bHI : 0.0, bHe1 = coll ? r.bHeI : 0.0, bHe2 = coll ? r.bHeII : 0.0;
  const double y1 = (1.0 - y2) - y3;
  const double ne = c.nH * x + c.nHe * (y2 + 2.0 * y3);
  const double GH = c.GH, G1 = c.G1, G2 = c.G2;
  // rates of change at the start of the sub-step (for the step size)
  const double IH = GH + bH * ne, RH = aH * ne;
  const double I1 = G1 + bHe1 * ne, R2 = aHe2 * ne, I2 = G2 + bHe2 * ne, R3 = aHe3 * ne;
  // constant sources (photon-conserving coupling), for the step size at most
  // what the atoms present can take over the time left.  With no source
  // (the default coupling) and a fraction that is not negative the cap is
  // min(0, v >= 0) = 0: the FP64 division is skipped, the value is the same
  double sH = (c.SH > 0.0 || (1.0 - x) < 0.0) ? fmin(c.SH, (1.0 - x) / rem) : 0.0;
  double s1 = (c.S1 > 0.0 || y1 < 0.0) ? fmin(c.S1, y1 / rem) : 0.0;
  double s2 = (c.S2 > 0.0 || y2 < 0.0) ? fmin(c.S2, y2 / rem) : 0.0;
  const double dx = (sH + IH * (1.0 - x)) - RH * x;
  const double dy1 = (-I1 * y1 + R2 * y2) - s1;
  const double dy3 = (s2 + I2 * y2) - R3 * y3;
  const double dy2 = -dy1 - dy3;
  double h = rem;
  {
    const double val[5] = {1.0 - x, x, y1, y2, y3};
    const double der[5] = {-dx, dx, dy1, dy2, dy3};
    const int nv = he ? 5 : 2;
    for (int i = 0; i < nv; ++i) {
      const double fl = val[i] > 1e-3 ? val[i] : 1e-3;
      const double ad = fabs(der[i]);
      if (ad * h > c.eps * fl) h = c.eps * fl / ad;
    }
  }
  const double ntot = c.nH + c.nHe + ne;
  if (!c.iso) {
    const double nHI = c.nH * (1.0 - x), nHII = c.nH * x;
    const double heat = (c.WH * nHI + c.W1 * (c.nHe * y1) + c.W2 * (c.nHe * y2)) + c.heat_rate;
    const double L = cooling_rate(r, c.mask, ne, nHI, nHII, c.nHe * y1, c.nHe * y2, c.nHe * y3) +
                     c.ccomp * ne * (T - c.Tcmb);
    const double dne = c.nH * dx + c.nHe * (dy2 + 2.0 * dy3);
    // (dT is only the step-size estimate: the reciprocal constant's rounding does not matter)
    const double dT = ((heat - L) * (1.0 / (1.5 * kB)) - T * dne) / ntot;
    const double adT = fabs(dT);
    if (adT * h > c.eps * T) h = c.eps * T / adT;
  }
  if (nsub == c.max_sub - 1 || !(h < rem)) h = rem;
  // the sources of the sub-step ionise at most the atoms present (He II also
  // what He I gives it): the photons beyond are lost
  sH = (c.SH > 0.0 || (1.0 - x) < 0.0) ? fmin(c.SH, (1.0 - x) / h) : 0.0;
  s1 = (c.S1 > 0.0 || y1 < 0.0) ? fmin(c.S1, y1 / h) : 0.0;
  s2 = (c.S2 > 0.0 || y2 < 0.0 || s1 < 0.0) ? fmin(c.S2, y2 / h + s1) : 0.0;
  // implicit ionisation update
  double xn = x, y1n = y1, y2n = y2, y3n = y3, nen = ne;
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    const double ih = GH + bH * nen, rh = aH * nen;
    const double xnum = x + h * (sH + ih), xden = 1.0 + h * (ih + rh);
    if (!he) xn = xnum / xden;
    if (he) {
      const double i1 = G1 + bHe1 * nen, r2 = aHe2 * nen;
      const double i2 = G2 + bHe2 * nen, r3 = aHe3 * nen;
      // tridiagonal (I - h Q) y_new = y_old, Thomas elimination
      const double a11 = 1.0 + h * i1, a12 = -h * r2;
      const double a21 = -h * i1, a22 = 1.0 + h * (r2 + i2), a23 = -h * r3;
      const double a32 = -h * i2, a33 = 1.0 + h * r3;
      // right-hand side: the old fractions plus the constant sources
      const double b1 = y1 - h * s1, b2 = y2 + h * (s1 - s2), b3 = y3 + h * s2;
      const double inv11 = 1.0 / a11;
      const double c1 = a12 * inv11, d1 = b1 * inv11;
      const double inv2 = 1.0 / (a22 - a21 * c1);
      const double c2 = a23 * inv2, d2 = (b2 - a21 * d1) * inv2;
      // the last elimination step and the H update share one division
      // (both denominators are at least 1)
      const double den3 = a33 - a32 * c2;
      const double r = 1.0 / (xden * den3);
      y3n = ((b3 - a32 * d2) * xden) * r;
      xn = (xnum * den3) * r;
      y2n = d2 - c2 * y3n;
      y1n = d1 - c1 * y2n;
    }
    const double ne_it = c.nH * xn + c.nHe * (y2n + 2.0 * y3n);
    const bool converged = fabs(ne_it - nen) <= 1e-12 * ne_it;
    nen = ne_it;
    if (converged) break;
  }
  xn = fmin(fmax(xn, 0.0), 1.0);
  if (he) {
    y1n = fmax(y1n, 0.0);
    y2n = fmax(y2n, 0.0);
    y3n = fmax(y3n, 0.0);
    const double inv_s = 1.0 / ((y1n + y2n) + y3n);
    y2n = y2n * inv_s;
    y3n = y3n * inv_s;
    y1n = (1.0 - y2n) - y3n;
  }
  const double ne2 = c.nH * xn + c.nHe * (y2n + 2.0 * y3n);
  if (!c.iso) {
    const double nHI = c.nH * (1.0 - xn), nHII = c.nH * xn;
    const double heat = (c.WH * nHI + c.W1 * (c.nHe * y1n) + c.W2 * (c.nHe * y2n)) + c.heat_rate;
    const double L = cooling_rate(r, c.mask, ne2, nHI, nHII, c.nHe * y1n, c.nHe * y2n,
                                  c.nHe * y3n);
    const double Cc = c.ccomp * ne2;
    const double ntot2 = c.nH + c.nHe + ne2;
    // semi-implicit cooling (linear in the new T): numerator and denominator
    // of the update taken times T, so that L / T needs no division of its own
    T = ((1.5 * kB * ntot * T + h * (heat + Cc * c.Tcmb)) * T) / ((1.5 * kB * ntot2 + h * Cc) * T + h * L);
  }
  if (COUNT && c.count_rec && rec) {
    nrec[0] += h * gH * ne2 * (c.nH * xn);
    if (he) {
      nrec[1] += h * g2 * ne2 * (c.nHe * y2n);
      nrec[2] += h * g3 * ne2 * (c.nHe * y3n);
    }
  }
  x = xn;
  y2 = y2n;
  y3 = y3n;
  rem = (h == rem) ? 0.0 : rem - h;
}


}  // namespace

// Per-cell inputs of the integration, from the step's deposits (Sec. 2
// coupling: photo-ionisation rate per frozen absorber, mean excess energy).
__device__ __forceinline__ void load_cell(const StepArgs& a, int64_t i, int b, CellIn& c, double& x,
                                          double& y2, double& y3, double& T) {
  const BoxMeta* M = a.boxes + b;
  const int E = a.box_E[b];
  const double q = ldexp(1.0, E);
  const double qE = ldexp(1.0, E + M->heatF) * eV;
  const double V = (M->dl * M->dl) * M->dl;
  x = a.xHII[i]; y2 = a.xHeII[i]; y3 = a.xHeIII[i]; T = a.T[i];
  c.nH = (double)a.nH[i];
  c.nHe = c.nH * M->he;
  const double NHI = (c.nH * (1.0 - x)) * V;
  const double NHeI = (c.nHe * ((1.0 - y2) - y3)) * V;
  const double NHeII = (c.nHe * y2) * V;
  const ulonglong2 d01 = reinterpret_cast<const ulonglong2*>(a.dep)[2 * i];
  const ulonglong2 d23 = reinterpret_cast<const ulonglong2*>(a.dep)[2 * i + 1];
  const long long dHI = (long long)d01.x, dHeI = (long long)d01.y;
  const long long dHeII = (long long)d23.x, dE = (long long)d23.y;
  c.SH = c.S1 = c.S2 = c.heat_rate = 0.0;
  if (!M->coupling) {
    c.GH = NHI > 0 ? ((double)dHI * q) / (a.dt * NHI) : 0.0;
    c.G1 = NHeI > 0 ? ((double)dHeI * q) / (a.dt * NHeI) : 0.0;
    c.G2 = NHeII > 0 ? ((double)dHeII * q) / (a.dt * NHeII) : 0.0;
    const long long nabs = (dHI + dHeI) + dHeII;
    const double eps_heat = nabs > 0 ? ((double)dE * qE) / ((double)nabs * q) : 0.0;
    c.WH = eps_heat * c.GH;
    c.W1 = eps_heat * c.G1;
    c.W2 = eps_heat * c.G2;
  } else {
    // photon-conserving: one ionisation per absorbed photon at a constant
    // rate per atom of the element, heating at the deposited rate
    const double NH = c.nH * V, NHe = c.nHe * V;
    c.GH = c.G1 = c.G2 = 0.0;
    c.WH = c.W1 = c.W2 = 0.0;
    c.SH = NH > 0 ? ((double)dHI * q) / (a.dt * NH) : 0.0;
    c.S1 = NHe > 0 ? ((double)dHeI * q) / (a.dt * NHe) : 0.0;
    c.S2 = NHe > 0 ? ((double)dHeII * q) / (a.dt * NHe) : 0.0;
    c.heat_rate = ((double)dE * qE) / (a.dt * V);
  }
  // the uniform background acts in every cell, whatever the deposits
  c.GH += M->uv[0];
  c.G1 += M->uv[1];
  c.G2 += M->uv[2];
  c.WH += M->uv[0] * (M->uve[0] * eV);
  c.W1 += M->uv[1] * (M->uve[1] * eV);
  c.W2 += M->uv[2] * (M->uve[2] * eV);
  c.iso = M->isothermal;
  // the diffuse recombination field replaces on-the-spot absorption: case A
  c.caseB = M->f_rec > 0.0 ? 0 : M->caseB;
  c.count_rec = M->f_rec > 0.0;
  c.V = V;
  c.Tcmb = M->T_cmb;
  c.mask = a.cool_mask;
  if (M->T_cmb > 0 && (a.cool_mask & 16)) {
    const double t2 = M->T_cmb * M->T_cmb;
    c.ccomp = 4.0 * sigmaT * aRad * (t2 * t2) * kB / (mE * cLight);
  } else {
    c.ccomp = 0.0;
  }
  c.eps = a.chem_eps;
  c.max_sub = a.chem_max_sub;
}

// Persistent kernel: every lane integrates one cell at a time, one sub-step
// per loop turn, and takes the next unclaimed cell (warp-aggregated atomic
// on a step counter) as soon as its cell is done.  Cells need from one to
// thousands of sub-steps, so handing out work per lane keeps the warps full
// instead of waiting for the slowest cell of a fixed group of 32.
template <typename RT, bool COUNT>
__global__ void __launch_bounds__(128) k_chemistry(StepArgs a, unsigned long long* next_cell) {
  const unsigned full = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const int64_t n = a.n_cells_total;
  int64_t i = -1;
  int b = -1, tb = -1;
  CellIn c;
  double x = 0, y2 = 0, y3 = 0, T = 0, rem = 0;
  int nsub = 0;
  unsigned long long subs = 0;
  double nrec[3] = {0.0, 0.0, 0.0};
  bool need = true, exhausted = false;
  while (true) {
    const unsigned m = __ballot_sync(full, need && !exhausted);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(next_cell, (unsigned long long)__popc(m));
      base = __shfl_sync(full, base, leader);
      if (need && !exhausted) {
        i = (int64_t)base + __popc(m & ((1u << lane) - 1u));
        if (i >= n) {
          exhausted = true;
          i = -1;
        } else {
          b = box_of_cell(a.boxes, a.n_boxes, i);
          if (b != tb) {
            if (tb >= 0 && subs) atomicAdd(a.budget + tb * 8 + 7, subs);
            tb = b;
            subs = 0;
          }
          load_cell(a, i, b, c, x, y2, y3, T);
          rem = a.dt;
          nsub = 0;
          if (COUNT) nrec[0] = nrec[1] = nrec[2] = 0.0;
          need = false;
        }
      }
    }
    const bool active = !need;
    if (!__any_sync(full, active)) break;
    if (active) {
      substep<RT, COUNT>(c, x, y2, y3, T, rem, nsub, nrec);
      ++nsub;
      if (!(rem > 0.0)) {
        a.xHII[i] = x;
        a.xHeII[i] = y2;
        a.xHeIII[i] = y3;
        a.T[i] = T;
        if (COUNT && c.count_rec)
          for (int sp = 0; sp < 3; ++sp) a.rec[(int64_t)sp * n + i] += nrec[sp] * c.V;
        subs += (unsigned long long)nsub;
        need = true;
      }
    }
  }
  if (tb >= 0 && subs) atomicAdd(a.budget + tb * 8 + 7, subs);
}

void launch_chemistry(const StepArgs& a, cudaStream_t s) {
  if (a.n_cells_total <= 0) return;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = std::min<int64_t>((a.n_cells_total + 127) / 128, (int64_t)sms * 8);
  cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s);
  if (a.any_rec) {
    if (a.fp32_rates) k_chemistry<float, true><<<(unsigned)blocks, 128, 0, s>>>(a, a.work);
    else k_chemistry<double, true><<<(unsigned)blocks, 128, 0, s>>>(a, a.work);
  } else {
    if (a.fp32_rates) k_chemistry<float, false><<<(unsigned)blocks, 128, 0, s>>>(a, a.work);
    else k_chemistry<double, false><<<(unsigned)blocks, 128, 0, s>>>(a, a.work);
  }
}
