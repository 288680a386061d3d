// kernels.cu -- CUDA kernels of the constrained Langevin time step
// (Paquay & Kusters, Algorithm 1 and Algorithm S1) for sm_103a.
//
// One step (md_step) is, in launch order:
//   pair          f^k = -grad V(x^k): truncated-shifted LJ (Eq. S1) over the
//                 27 neighbour cells, harmonic bonds and walls (SI S3.2)
//   integrate     Algorithm S1 force combination with Philox noise, the
//                 momentum half of step k and the position half of step k+1
//                 (Algorithm 1), then the cell of x^{k+1} and its bucket rank
//   scan          exclusive scan of the bucket counters (one pass)
//   scatter       particles to their bucket slots
//   bucket build  canonical (particle-id) order inside each bucket and the
//                 cell-relative records the pair kernel reads
// The momentum half of step k and the position half of step k+1 share one
// kernel: between steps the state is (x^k, p^{k-1/2}) and the combined force
// never leaves registers; p^k is rebuilt on demand (launch_finish).
#include <algorithm>
#include <cfloat>
#include <type_traits>
#include <cmath>

#include "df.cuh"
#include "engine.h"

namespace surfmd {


// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products with the published multipliers; the key is bumped
// by the published Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Three normals of particle pid at step k: key (seed, replica), counter
// (pid, k_lo, k_hi, 0); Box-Muller on words (0,1) -> x, y and (2,3) -> z
// (cosine branch); u = ((w >> 9) + 1/2) 2^-23 is exact in float and double.
// Float32 (the mixed path's Langevin noise): the logarithm, sine and cosine
// are the hardware's fast approximations (absolute error about 1e-6 in a
// normal; the angle is taken as 2 pi (u - 1/2) in (-pi, pi), where their
// error bound holds, with the signs of sin and cos of 2 pi u restored). The
// float64 path (below) keeps the library functions: it matches the oracle's
// normals to rounding.
#ifndef SURFMD_FAST_NOISE
#define SURFMD_FAST_NOISE 1
#endif
__device__ __forceinline__ void gauss3(uint32_t seed, uint32_t rep, uint32_t pid, uint64_t k,
                                       float& gx, float& gy, float& gz) {
  const uint4 w = philox4x32_10(make_uint4(pid, (uint32_t)k, (uint32_t)(k >> 32), 0u),
                                make_uint2(seed, rep));
  const float s = 1.0f / 8388608.0f;
  const float u0 = ((float)(w.x >> 9) + 0.5f) * s, u1 = ((float)(w.y >> 9) + 0.5f) * s;
  const float u2 = ((float)(w.z >> 9) + 0.5f) * s, u3 = ((float)(w.w >> 9) + 0.5f) * s;
#if SURFMD_FAST_NOISE
  const float two_pi = 6.28318530717958648f;
  // (near u = 1 the fast logarithm's absolute error can exceed -ln u: clamp at 0)
  const float r01 = sqrtf(fmaxf(-2.0f * __logf(u0), 0.0f));
  const float r23 = sqrtf(fmaxf(-2.0f * __logf(u2), 0.0f));
  float sn, cs;
  __sincosf(two_pi * (u1 - 0.5f), &sn, &cs);
  gx = -r01 * cs;
  gy = -r01 * sn;
  gz = -r23 * __cosf(two_pi * (u3 - 0.5f));
#else
  const float r01 = sqrtf(-2.0f * logf(u0));
  const float r23 = sqrtf(-2.0f * logf(u2));
  float sn, cs;
  sincospif(2.0f * u1, &sn, &cs);
  gx = r01 * cs;
  gy = r01 * sn;
  gz = r23 * cospif(2.0f * u3);
#endif
}

__device__ __forceinline__ void gauss3(uint32_t seed, uint32_t rep, uint32_t pid, uint64_t k,
                                       double& gx, double& gy, double& gz) {
  const uint4 w = philox4x32_10(make_uint4(pid, (uint32_t)k, (uint32_t)(k >> 32), 0u),
                                make_uint2(seed, rep));
  const double s = 1.0 / 8388608.0;
  const double u0 = ((double)(w.x >> 9) + 0.5) * s, u1 = ((double)(w.y >> 9) + 0.5) * s;
  const double u2 = ((double)(w.z >> 9) + 0.5) * s, u3 = ((double)(w.w >> 9) + 0.5) * s;
  const double r01 = sqrt(-2.0 * log(u0));
  const double r23 = sqrt(-2.0 * log(u2));
  double sn, cs;
  sincospi(2.0 * u1, &sn, &cs);
  gx = r01 * cs;
  gy = r01 * sn;
  gz = r23 * cospi(2.0 * u3);
}

// Format conversions on the integer pipe. On this GPU a float64 <-> float32
// conversion issues on the float64 pipe at the float64 rate (two lanes per SM
// per clock), as costly as a DFMA; the mixed integrator converts a dozen
// values per particle. These build the result from the IEEE 754 binary64 and
// binary32 bit fields (sign, biased exponent with bias 1023 / 127, fraction of
// 52 / 23 bits) with integer operations. Zero and every normal binary32 result
// are formed here; binary32 subnormal results, overflow, infinities and NaN
// take the hardware conversion, so the result is bit-identical to it always.
//
// binary64 -> binary32, round to nearest, ties to even, with 32-bit integer
// operations on the two words of the binary64 value: the high word's
// exponent and fraction bits shifted up by 3 with the top 3 bits of the low
// word shifted in give (exponent << 23 | top 23 fraction bits) modulo 2^32;
// rebiasing subtracts 896 << 23; the 29 dropped bits round it (half-way cases
// to the even result), and a carry out of the fraction moves into the
// exponent, as rounding up to the next binade must.
__device__ __forceinline__ uint32_t d2f_bits_rn(uint32_t hi, uint32_t lo, uint32_t& up, uint32_t& rest) {
  const uint32_t t = __funnelshift_l(lo, hi & 0x7fffffffu, 3) - 0xC0000000u;  // 896 << 23 modulo 2^32
  rest = lo & 0x1fffffffu;
  up = (rest + (t & 1u) + 0x0fffffffu) >> 29;
  return t + up;
}

__device__ __forceinline__ float d2f_rn(double v) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  // biased binary64 exponent in [897, 1150] <=> binary32 exponent in [1, 254]
  if (((hi >> 20) & 0x7ffu) - 897u < 254u) {
    uint32_t up, rest;
    return __uint_as_float((hi & 0x80000000u) | d2f_bits_rn(hi, lo, up, rest));
  }
  if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi);
  return __double2float_rn(v);
}

// binary32 -> binary64 (exact): exponent + 896, fraction shifted up by 29.
__device__ __forceinline__ double f2d(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0x000fffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)v;
}

// float64 -> double-float on the integer pipe: h = v rounded to float32 (as
// d2f_rn), l = the remainder v - h. The remainder is an integer number rem of
// units 2^(E-1075) of v's binade (E = v's biased exponent; rem is the low
// bits of the fraction field minus the rounding, |rem| <= 2^28); l keeps its
// leading bits, rem >> 6 (<= 2^22 in magnitude, so converted exactly by the
// 1.5 * 2^23 bias), times 2^(E-1069). h + l = v within 2^-46 |v|. Outside
// 2^-80 <= |v| < 2^128 (zero, tiny or huge values) the split takes one
// float64 subtraction instead.
__device__ __forceinline__ DF df_from(double v) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 943u < 208u) {  // biased exponent in [943, 1150]
    uint32_t up, rest;
    const uint32_t q = d2f_bits_rn(hi, lo, up, rest);
    const int32_t rem = (int32_t)rest - (int32_t)(up << 29);  // dropped bits, less 2^29 if rounded up
    const float k = __fsub_rn(__int_as_float(0x4B400000 + (rem >> 6)), 12582912.0f);
    const float l = __fmul_rn(k, __uint_as_float((e - 942u) << 23));
    const uint32_t sign = hi & 0x80000000u;
    return {__uint_as_float(sign | q), sign ? -l : l};
  }
  const float h = d2f_rn(v);
  return {h, d2f_rn(v - f2d(h))};
}
__device__ __forceinline__ double df_to(DF a) { return f2d(a.h) + f2d(a.l); }

// ---------------------------------------------------------------------------
// Surfaces: g(x) and n = grad g (unnormalised), float64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double wrap_min_image(double d, double L) { return d - L * rint(d / L); }

// Thylakoid composite (SI S3.1), p = (R_b, L_x, R_c, L_b), centre c, z
// periodic: a bridge cylinder of radius R_b along x through (c_y, c_z) for
// |x - c_x| <= L_b/2; at each end a connector (tube radius R_c) meeting it
// and the face plane of a block at x = c_x -/+ (L_b/2 + R_c) with continuous
// tangent planes; each block a tube along z with a square cross section of
// side L_x + 2 R_c whose corners are quarter cylinders of radius R_c. A
// particle's piece is chosen from the position where its half step starts
// and held for that solve: between the block faces and within R_b + R_c of
// the bridge axis the bridge or the nearer connector, otherwise the block's
// rounded square (a corner cylinder beyond the inner square in x and y, else
// the plane of the side it lies beyond, the nearest side when inside), the
// face plane's hole belonging to the connector.
struct Piece {
  int type;  // 0 plane normal to x, 1 plane normal to y, 2 cylinder along z, 3 bridge, 4 connector
  double s, c0, c1, rad;
};

__device__ __forceinline__ double thyl_dz(const SysDev& S, double z) {
  const double d = z - S.c[2];
  return S.periodic[2] ? wrap_min_image(d, S.box_len[2]) : d;
}

__device__ __forceinline__ Piece thyl_select(const SysDev& S, double x, double y, double z) {
  const double Rb = S.p[0], Lx = S.p[1], Rc = S.p[2], Lb = S.p[3];
  const double xc = S.c[0], yc = S.c[1];
  const double x0L = xc - 0.5 * Lb, x0R = xc + 0.5 * Lb, xfL = x0L - Rc, xfR = x0R + Rc;
  const double dy = y - yc, dz = thyl_dz(S, z);
  const double r = sqrt(dy * dy + dz * dz), Rout = Rb + Rc;
  Piece q{0, 1.0, 0.0, 0.0, 0.0};
  if (x > xfL && x < xfR && r < Rout) {
    if (x < x0L) { q.type = 4; q.c0 = x0L; }
    else if (x > x0R) { q.type = 4; q.c0 = x0R; }
    else { q.type = 3; q.rad = Rb; }
    return q;
  }
  const bool left = x <= xc;
  const double ixl = left ? xfL - Rc - Lx : xfR + Rc, ixh = ixl + Lx;
  const double iyl = yc - 0.5 * Lx, iyh = yc + 0.5 * Lx;
  double ex = x < ixl ? x - ixl : (x > ixh ? x - ixh : 0.0);
  double ey = y < iyl ? y - iyl : (y > iyh ? y - iyh : 0.0);
  if (ex != 0.0 && ey != 0.0) {
    q.type = 2; q.c0 = ex < 0.0 ? ixl : ixh; q.c1 = ey < 0.0 ? iyl : iyh; q.rad = Rc;
    return q;
  }
  if (ex == 0.0 && ey == 0.0) {  // inside: the nearest side
    const double dxl = x - (ixl - Rc), dxh = (ixh + Rc) - x, dyl = y - (iyl - Rc), dyh = (iyh + Rc) - y;
    const double mx = dxl < dxh ? dxl : dxh, my = dyl < dyh ? dyl : dyh;
    if (mx <= my) ex = dxl < dxh ? -1.0 : 1.0;
    else ey = dyl < dyh ? -1.0 : 1.0;
  }
  if (ex != 0.0) {
    const bool face = left ? ex > 0.0 : ex < 0.0;  // the side that faces the bridge
    if (face && r < Rout) { q.type = 4; q.c0 = left ? x0L : x0R; return q; }
    q.type = 0; q.s = ex < 0.0 ? -1.0 : 1.0; q.c0 = ex < 0.0 ? ixl - Rc : ixh + Rc;
    return q;
  }
  q.type = 1; q.s = ey < 0.0 ? -1.0 : 1.0; q.c0 = ey < 0.0 ? iyl - Rc : iyh + Rc;
  return q;
}

// g and grad g of one piece at (x, y, z).
__device__ __forceinline__ double thyl_eval(const SysDev& S, const Piece& q, double x, double y, double z,
                                            double& nx, double& ny, double& nz) {
  const double Rc = S.p[2], Rout = S.p[0] + Rc;
  const double dy = y - S.c[1], dz = thyl_dz(S, z);
  switch (q.type) {
    case 0: nx = q.s; ny = 0.0; nz = 0.0; return q.s * (x - q.c0);
    case 1: nx = 0.0; ny = q.s; nz = 0.0; return q.s * (y - q.c0);
    case 2: {
      const double a = x - q.c0, b = y - q.c1;
      nx = 2.0 * a; ny = 2.0 * b; nz = 0.0;
      return a * a + b * b - q.rad * q.rad;
    }
    case 3:
      nx = 0.0; ny = 2.0 * dy; nz = 2.0 * dz;
      return dy * dy + dz * dz - q.rad * q.rad;
    default: {
      const double r = sqrt(dy * dy + dz * dz), a = x - q.c0, t = r - Rout;
      const double w = 2.0 * (1.0 - Rout / r);
      nx = 2.0 * a; ny = w * dy; nz = w * dz;
      return a * a + t * t - Rc * Rc;
    }
  }
}

__device__ __forceinline__ double surf_eval(const SysDev& S, double x, double y, double z,
                                            double& nx, double& ny, double& nz) {
  double dx = x - S.c[0], dy = y - S.c[1], dz = z - S.c[2];
  switch (S.kind) {
    case kPlane:
      nx = S.p[0]; ny = S.p[1]; nz = S.p[2];
      return fma(S.p[0], dx, fma(S.p[1], dy, S.p[2] * dz));
    case kSphere:
      nx = 2.0 * dx; ny = 2.0 * dy; nz = 2.0 * dz;
      return fma(dx, dx, fma(dy, dy, fma(dz, dz, -S.p[0] * S.p[0])));
    case kEllipsoid: {
      const double ax = dx * S.inv_a2[0], ay = dy * S.inv_a2[1], az = dz * S.inv_a2[2];
      nx = 2.0 * ax; ny = 2.0 * ay; nz = 2.0 * az;
      return fma(ax, dx, fma(ay, dy, fma(az, dz, -1.0)));
    }
    case kTorus: {
      const double rho = sqrt(fma(dx, dx, dy * dy));
      const double t = rho - S.p[0];
      const double q = 2.0 * t / rho;
      nx = q * dx; ny = q * dy; nz = 2.0 * dz;
      return fma(t, t, fma(dz, dz, -S.p[1] * S.p[1]));
    }
    case kBump: {
      if (S.periodic[0]) dx = wrap_min_image(dx, S.box_len[0]);
      if (S.periodic[1]) dy = wrap_min_image(dy, S.box_len[1]);
      const double w2 = S.p[1] * S.p[1];
      const double e = S.p[0] * exp(-fma(dx, dx, dy * dy) / (2.0 * w2));
      nx = e * dx / w2; ny = e * dy / w2; nz = 1.0;
      return dz - e;
    }
    case kCylinder: {
      const int ax = S.axis;
      if (ax == 0) dx = 0.0;
      else if (ax == 1) dy = 0.0;
      else dz = 0.0;
      nx = 2.0 * dx; ny = 2.0 * dy; nz = 2.0 * dz;
      return fma(dx, dx, fma(dy, dy, fma(dz, dz, -S.p[0] * S.p[0])));
    }
    case kThylakoid: {  // the piece at the point itself
      const Piece q = thyl_select(S, x, y, z);
      return thyl_eval(S, q, x, y, z, nx, ny, nz);
    }
    default:
      nx = ny = nz = 0.0;
      return 0.0;
  }
}

// ---------------------------------------------------------------------------
// Cell grid
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bucket_of(uint32_t cell, int hashed, int log_t) {
  if (!hashed) return cell;
  const uint32_t h = ((cell >> 3) * 0x9E3779B1u) >> (35 - log_t);
  return (h << 3) | (cell & 7u);
}

// Coordinate wrapped into the periodic box (unchanged on open axes). The
// binning arithmetic is written with round-to-nearest intrinsics (no FMA
// contraction) so that the cell of a particle is reproducible on the host.
__device__ __forceinline__ double wrap_coord(const SysDev& S, int d, double v) {
  if (!S.periodic[d]) return v;
  const double L = S.box_len[d];
  const double r = __dsub_rn(v, S.box_lo[d]);
  return __dadd_rn(S.box_lo[d], __dsub_rn(r, __dmul_rn(L, floor(__ddiv_rn(r, L)))));
}

__device__ __forceinline__ int cell_coord(const SysDev& S, int d, double v, bool& out) {
  const double t = __dmul_rn(__dsub_rn(v, S.grid_lo[d]), S.inv_cs[d]);
  int c = (int)floor(t);
  if (c < 0) {
    if (!S.periodic[d]) out = true;
    c = 0;
  } else if (c >= S.nc[d]) {
    if (!S.periodic[d] || c > S.nc[d]) out = true;
    c = S.nc[d] - 1;
  }
  if (!(t == t)) {
    out = true;
    c = 0;
  }
  return c;
}

__device__ __forceinline__ uint32_t cell_id(const SysDev& S, int cx, int cy, int cz) {
  return S.cell_base + (uint32_t)cx + (uint32_t)S.nc[0] * ((uint32_t)cy + (uint32_t)S.nc[1] * (uint32_t)cz);
}

// Cell of a position, float64 binning (float64 path).
__device__ __forceinline__ uint32_t cell_of_d(const SysDev& S, double x, double y, double z, bool& out) {
  const int cx = cell_coord(S, 0, wrap_coord(S, 0, x), out);
  const int cy = cell_coord(S, 1, wrap_coord(S, 1, y), out);
  const int cz = cell_coord(S, 2, wrap_coord(S, 2, z), out);
  return cell_id(S, cx, cy, cz);
}

// Cell of a position, float32 binning (mixed path): the coordinate is rounded
// to float, wrapped and scaled in float with round-to-nearest intrinsics. The
// cell edge carries a 2^-12 margin over the cutoff, far more than the float
// rounding of a coordinate, so a neighbour within the cutoff is still at most
// one cell away.
__device__ __forceinline__ int cell_coord_f(const SysDev& S, int d, double v, bool& out) {
  float u = d2f_rn(v);
  if (S.periodic[d]) {
    const float L = S.box_len_f[d];
    const float r = __fsub_rn(u, S.box_lo_f[d]);
    u = __fadd_rn(S.box_lo_f[d], __fsub_rn(r, __fmul_rn(L, floorf(__fdiv_rn(r, L)))));
  }
  const float t = __fmul_rn(__fsub_rn(u, S.grid_lo_f[d]), S.inv_cs_f[d]);
  int c = (int)floorf(t);
  if (c < 0) {
    if (!S.periodic[d]) out = true;
    c = 0;
  } else if (c >= S.nc[d]) {
    if (!S.periodic[d] || c > S.nc[d]) out = true;
    c = S.nc[d] - 1;
  }
  if (!(t == t)) {
    out = true;
    c = 0;
  }
  return c;
}

__device__ __forceinline__ uint32_t cell_of_f(const SysDev& S, double x, double y, double z, bool& out) {
  return cell_id(S, cell_coord_f(S, 0, x, out), cell_coord_f(S, 1, y, out), cell_coord_f(S, 2, z, out));
}

template <typename R>
__device__ __forceinline__ uint32_t cell_of(const SysDev& S, double x, double y, double z, bool& out) {
  return sizeof(R) == 4 ? cell_of_f(S, x, y, z, out) : cell_of_d(S, x, y, z, out);
}

__device__ __forceinline__ void cell_decode(const SysDev& S, uint32_t cell, int& cx, int& cy, int& cz) {
  uint32_t r = cell - S.cell_base;
  cx = (int)(r % (uint32_t)S.nc[0]);
  r /= (uint32_t)S.nc[0];
  cy = (int)(r % (uint32_t)S.nc[1]);
  cz = (int)(r / (uint32_t)S.nc[1]);
}

__device__ __forceinline__ void flag(uint32_t* status, uint32_t bit) { atomicOr(status, bit); }

__device__ __forceinline__ bool finite3(double a, double b, double c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

// ---------------------------------------------------------------------------
// meta / set state / restore
// ---------------------------------------------------------------------------
__global__ void k_build_meta(DevArrays A, const int64_t* __restrict__ first, int nsys,
                             const int32_t* __restrict__ type, const uint8_t* __restrict__ con,
                             const int32_t* __restrict__ mol) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int lo = 0, hi = nsys - 1;  // last system with first <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= i) lo = mid; else hi = mid - 1;
  }
  const SysDev& S = A.sys[lo];
  int t = type ? type[i] : 0;
  if (t < 0 || t >= A.ntypes) {
    flag(A.status, kFlagOffSurface);
    t = 0;
  }
  // the unconstrained 2D plane holds no particle by a constraint
  const uint32_t c = S.kind == kXY2D ? 0u : (con ? (con[i] ? 1u : 0u) : (S.kind != kNone ? 1u : 0u));
  A.meta[i] = meta_pack((uint32_t)t, (S.kind != kNone) ? c : 0u, (uint32_t)lo);
  if (S.kind != kNone && !c) atomicAdd(&A.sys_free[lo], 1);
  if (A.mol) {
    const int64_t pid = i - S.first;
    A.mol[i] = mol ? mol[i] : (int32_t)(S.bpm > 1 ? pid / S.bpm : pid);
  }
}

__global__ void k_set_state(DevArrays A, const double* __restrict__ xa, const double* __restrict__ va) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (i >= n) return;
  const uint32_t m = A.meta[i];
  const SysDev& S = A.sys[meta_sys(m)];
  const double x = xa[3 * i], y = xa[3 * i + 1], z = xa[3 * i + 2];
  double vx = va ? va[3 * i] : 0.0, vy = va ? va[3 * i + 1] : 0.0, vz = va ? va[3 * i + 2] : 0.0;
  if (!finite3(x, y, z) || !finite3(vx, vy, vz)) flag(A.status, kFlagOffSurface);
  if (S.kind == kXY2D) {  // in the plane z = c_z, no motion along z
    if (!(fabs(z - S.c[2]) < 1e-6)) flag(A.status, kFlagOffSurface);
    vz = 0.0;
  }
  if (meta_con(m)) {
    double nx, ny, nz;
    const double g = surf_eval(S, x, y, z, nx, ny, nz);
    const double n2 = nx * nx + ny * ny + nz * nz;
    if (!(fabs(g) < 1e-6 * sqrt(n2))) flag(A.status, kFlagOffSurface);
    const double s = (nx * vx + ny * vy + nz * vz) / n2;
    vx -= s * nx; vy -= s * ny; vz -= s * nz;
  }
  const double mass = A.types->mass[meta_type(m)];
  A.x[i] = x; A.x[n + i] = y; A.x[2 * n + i] = z;
  A.xref[i] = x; A.xref[n + i] = y; A.xref[2 * n + i] = z;
  A.ph[i] = mass * vx; A.ph[n + i] = mass * vy; A.ph[2 * n + i] = mass * vz;
  A.pk[i] = mass * vx; A.pk[n + i] = mass * vy; A.pk[2 * n + i] = mass * vz;
}

__global__ void k_restore(DevArrays A, const double* __restrict__ xa, const double* __restrict__ pa) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (i >= n) return;
  for (int d = 0; d < 3; ++d) {
    A.x[d * n + i] = xa[3 * i + d];
    A.ph[d * n + i] = pa[3 * i + d];
  }
  if (!finite3(xa[3 * i], xa[3 * i + 1], xa[3 * i + 2])) flag(A.status, kFlagNonfinite);
}

// ---------------------------------------------------------------------------
// cell list
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void bin_one(const DevArrays& A, int64_t i) {
  const int64_t n = A.n;
  const SysDev& S = A.sys[meta_sys(A.meta[i])];
  bool out = false;
  const uint32_t cell = cell_of<R>(S, A.x[i], A.x[n + i], A.x[2 * n + i], out);
  if (out) flag(A.status, kFlagOutOfGrid);
  A.cell[i] = cell;
  A.rank[i] = atomicAdd(&A.count[bucket_of(cell, A.hashed, A.log_t)], 1u);
}

template <typename R>
__global__ void k_bin(DevArrays A) {
  if (A.nl_dirty && *A.nl_dirty == 0u) return;  // neighbour-list mode, no rebuild this step
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.n) bin_one<R>(A, i);
}

constexpr int kScanThreads = 512;
constexpr int kScanItems = kScanPerBlock / kScanThreads;  // 16 (four uint4)

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t& block_total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? warp_tot[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) warp_tot[lane] = wi - w;
    if (lane == nw - 1) warp_tot[32] = wi;
  }
  __syncthreads();
  block_total = warp_tot[32];
  return warp_tot[wid] + inc - v;
}

// Exclusive scan of the bucket counters in one pass (decoupled look-back):
// each CTA takes the next tile index from a counter (so every tile's
// predecessors have started), scans its kScanPerBlock counters, publishes its
// aggregate, then walks back over its predecessors' published values until it
// meets an inclusive prefix. Tile states are 64-bit words
// (epoch:30 | flag:2 | value:32); a state from an earlier launch (older epoch)
// reads as "not ready". Every wait is bounded: a predecessor's word is read at
// most A.spin_limit times; if it is still not ready the kernel sets the
// timeout flag and takes a zero prefix for its tile, so every bucket start
// stays within [0, n] (the list is wrong, every later access stays in bounds,
// and the host rebuilds the list before the next step). The last CTA to
// finish resets the tile counter and advances the epoch. Optionally the
// kernel also moves the step counter on (nothing in it reads the step).
constexpr uint32_t kTileAgg = 1u, kTileIncl = 2u;

__device__ __forceinline__ unsigned long long tile_word(uint32_t epoch, uint32_t flag, uint32_t value) {
  return ((unsigned long long)(epoch & 0x3fffffffu) << 34) | ((unsigned long long)flag << 32) | value;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_onepass(DevArrays A, int advance) {
  __shared__ uint32_t warp_tot[33];
  __shared__ uint32_t s_tile, s_prefix;
  uint32_t* __restrict__ count = A.count;
  const uint32_t T = A.nbucket;
  ScanCtl* ctl = A.scan;
  const uint32_t epoch = ctl->epoch;
  if (A.nl_dirty && *A.nl_dirty == 0u) {  // neighbour-list mode, no rebuild: only the step advance
    if (threadIdx.x == 0 && atomicAdd(&ctl->done, 1u) == gridDim.x - 1) {
      ctl->done = 0u;
      if (advance) {
        if (A.nl_dirty && A.noise_k) *A.noise_k = *A.step;  // list mode: this step's normals are stored
        *A.step += 1ull;
        *A.mode = 1;
      }
    }
    return;
  }
  if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->tile, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t base = tile * (uint32_t)kScanPerBlock + threadIdx.x * kScanItems;
  const bool full = base + kScanItems <= T;  // whole run in range: 16-byte vector accesses
  uint32_t v[kScanItems];
  if (full) {
#pragma unroll
    for (int j = 0; j < kScanItems; j += 4) {
      const uint4 q = *reinterpret_cast<const uint4*>(count + base + j);
      v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) v[j] = (base + j < T) ? count[base + j] : 0u;
  }
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) sum += v[j];
  uint32_t total;
  const uint32_t excl = block_exclusive_scan(sum, warp_tot, total);
  if (threadIdx.x < 32) {  // warp 0 publishes and looks back 32 predecessors per probe
    volatile unsigned long long* st = A.tile_state;
    const int lane = threadIdx.x;
    const uint32_t ep = epoch & 0x3fffffffu;
    uint32_t prefix = 0;
    if (tile == 0) {
      if (lane == 0) st[0] = tile_word(epoch, kTileIncl, total);
    } else {
      if (lane == 0) st[tile] = tile_word(epoch, kTileAgg, total);
      __threadfence();
      int32_t hi = (int32_t)tile - 1;  // highest predecessor not yet summed
      bool timed_out = false;
      while (hi >= 0) {
        const int32_t j = hi - lane;
        unsigned long long w = 0ull;
        uint32_t flag = kTileIncl;  // lanes beyond tile 0 act as an empty inclusive prefix
        if (j >= 0) {
          // ready: written in this launch (epoch) with a flag (zeroed words carry none)
          bool ready = false;
          for (uint32_t reads = 0; reads < A.spin_limit && !ready; ++reads) {
            w = st[j];
            ready = (uint32_t)(w >> 34) == ep && ((w >> 32) & 3u) != 0u;
          }
          if (!ready) timed_out = true;
          flag = (uint32_t)((w >> 32) & 3u);
        }
        // the nearest inclusive prefix among the 32 (lowest lane holding one)
        const unsigned incl = __ballot_sync(0xffffffffu, flag == kTileIncl);
        const int stop = incl ? __ffs(incl) - 1 : 32;  // lanes 0..stop contribute
        uint32_t part = (lane <= stop && j >= 0) ? (uint32_t)w : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (__any_sync(0xffffffffu, timed_out)) {  // give up: a zero prefix keeps the starts in [0, n]
          if (lane == 0) atomicOr(A.status, kFlagTimeout);
          prefix = 0;
          break;
        }
        prefix += part;
        if (incl) break;
        hi -= 32;
      }
      __threadfence();
      if (lane == 0) st[tile] = tile_word(epoch, kTileIncl, prefix + total);
    }
    if (lane == 0) s_prefix = prefix;
  }
  __syncthreads();
  uint32_t run = excl + s_prefix;
  if (full) {
#pragma unroll
    for (int j = 0; j < kScanItems; j += 4) {
      uint4 o;
      o.x = run; run += v[j];
      o.y = run; run += v[j + 1];
      o.z = run; run += v[j + 2];
      o.w = run; run += v[j + 3];
      *reinterpret_cast<uint4*>(A.start + base + j) = o;
      *reinterpret_cast<uint4*>(count + base + j) = make_uint4(0u, 0u, 0u, 0u);
    }
  } else {
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
      if (base + j < T) {
        A.start[base + j] = run;
        run += v[j];
        count[base + j] = 0u;
      }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t nblk = gridDim.x;
    if (atomicAdd(&ctl->done, 1u) == nblk - 1) {  // last CTA: reset for the next launch
      ctl->done = 0u;
      ctl->tile = 0u;
      ctl->epoch = epoch + 1u;
      if (advance) {
        if (A.nl_dirty && A.noise_k) *A.noise_k = *A.step;  // list mode: this step's normals are stored
        *A.step += 1ull;
        *A.mode = 1;
      }
    }
  }
}

__device__ __forceinline__ void scatter_one(const DevArrays& A, int64_t i) {
  const uint32_t b = bucket_of(A.cell[i], A.hashed, A.log_t);
  A.stag_tmp[A.start[b] + A.rank[i]] = (uint32_t)i;
}

__global__ void k_scatter(DevArrays A) {
  if (A.nl_dirty && *A.nl_dirty == 0u) return;  // neighbour-list mode, no rebuild this step
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.n) scatter_one(A, i);
}

// Record of slot s. Mixed path: the offset rounded to float32 (the high
// part) and the remainder (the low part, in lo[s]); float64 path: the offset.
template <typename R> __device__ __forceinline__ void put_rec(void* rec, float4* lo, uint32_t s, double ox,
                                                              double oy, double oz, uint32_t bits);
template <> __device__ __forceinline__ void put_rec<float>(void* rec, float4* lo, uint32_t s, double ox,
                                                           double oy, double oz, uint32_t bits) {
  const DF x = df_from(ox), y = df_from(oy), z = df_from(oz);
  reinterpret_cast<float4*>(rec)[s] = make_float4(x.h, y.h, z.h, __uint_as_float(bits));
  lo[s] = make_float4(x.l, y.l, z.l, 0.f);
}
template <> __device__ __forceinline__ void put_rec<double>(void* rec, float4*, uint32_t s, double ox, double oy,
                                                            double oz, uint32_t bits) {
  reinterpret_cast<double4_32a*>(rec)[s] =
      make_double4_32a(ox, oy, oz, __longlong_as_double((long long)bits));
}

// Offset of a position from the centre of its cell, formed in float64 (the
// records store it in float32 on the mixed path: |o| <= cs/2 keeps its
// rounding small).
__device__ __forceinline__ void cell_offsets(const SysDev& S, uint32_t cell, double x, double y, double z,
                                             double o[3]) {
  int c[3];
  cell_decode(S, cell, c[0], c[1], c[2]);
  const double xv[3] = {x, y, z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // offset from the cell centre: |o| <= cs/2 keeps float32 rounding small
    // c + 1/2 is exact in float32 (c < 2^22), so the centre is the same float64 value either way
    o[k] = xv[k] - fma(f2d((float)c[k] + 0.5f), S.cs[k], S.grid_lo[k]);
    // the image the binning chose. With three or more cells on the axis, o lies within cs/2 <= L/6 of a
    // multiple of the box length L, far from an odd multiple of L/2, so o / L and o * (1 / L) round to
    // the same integer and the reciprocal form (no float64 divide) picks the same image.
    if (S.periodic[k])
      o[k] = S.nc[k] >= 3 ? fma(-S.box_len[k], rint(o[k] * S.inv_box_len[k]), o[k])
                          : wrap_min_image(o[k], S.box_len[k]);
  }
}

// One thread per slot: a particle's place inside its bucket is the number of
// bucket members with a smaller id, which gives every bucket one canonical
// order (so every force sum has one fixed order and runs repeat bit for bit).
// The thread writes the slot's particle id, cell id and its offset from the
// cell centre (formed in float64, stored in R).
template <typename R>
__device__ __forceinline__ void bucket_build_one(const DevArrays& A, int64_t s) {
  const int64_t n = A.n;
  const uint32_t tag = A.stag_tmp[s];
  const uint32_t cell = A.cell[tag];
  const uint32_t b = bucket_of(cell, A.hashed, A.log_t);
  const uint32_t s0 = A.start[b], s1 = A.start[b + 1];
  uint32_t rank = 0;
  for (uint32_t t = s0; t < s1; ++t) rank += (A.stag_tmp[t] < tag) ? 1u : 0u;
  const uint32_t d = s0 + rank;
  if (d >= (uint32_t)n) return;  // only after a scan that timed out (its starts are not a partition)
  const uint32_t m = A.meta[tag];
  const SysDev& S = A.sys[meta_sys(m)];
  double o[3];
  cell_offsets(S, cell, A.x[tag], A.x[n + tag], A.x[2 * n + tag], o);
  const uint32_t mol = A.mol ? (uint32_t)A.mol[tag] : 0u;
  A.stag[d] = tag;
  A.scell[d] = cell;
  if (A.slot_of) A.slot_of[tag] = d;
  if (A.smeta) A.smeta[d] = m;
  put_rec<R>(A.rec, A.rec_lo, d, o[0], o[1], o[2], meta_type(m) | ((A.rec_cell ? cell : mol) << 3));
}

template <typename R>
__global__ void k_bucket_build(DevArrays A) {
  if (A.nl_dirty && *A.nl_dirty == 0u) return;  // neighbour-list mode, no rebuild this step
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < A.n) bucket_build_one<R>(A, s);
}

// float64 reciprocal and inverse square root without the long divide/sqrt
// sequences: a float32 hardware estimate refined by Newton-Raphson steps
// (Newton's method on 1/e - v = 0 and on 1/e^2 - v = 0), each step doubling
// the correct bits (2^-22 -> 2^-44 -> full float64). v must be a positive
// normal number inside the float32 range; otherwise the float64 operator is
// used.
__device__ __forceinline__ double nr_rcp(double v) {
  const float vf = d2f_rn(v);
  if (!(vf > 1.0e-37f && vf < 1.0e37f)) return 1.0 / v;
  double e = f2d(__frcp_rn(vf));
  e = fma(e, fma(-v, e, 1.0), e);
  e = fma(e, fma(-v, e, 1.0), e);
  return e;
}

__device__ __forceinline__ double nr_rsqrt(double v) {
  const float vf = d2f_rn(v);
  if (!(vf > 1.0e-37f && vf < 1.0e37f)) return 1.0 / sqrt(v);
  double r = f2d(rsqrtf(vf));
  const double hv = 0.5 * v;
  r = r * fma(-hv * r, r, 1.5);
  r = r * fma(-hv * r, r, 1.5);
  return r;
}

// Surface direction in float32 (mixed path): the gradient of g at a point
// whose offset from the surface centre is (dx, dy, dz). Only the direction of
// n enters the position half (x = y - a lambda n) and the projection; a float
// direction moves the correction a lambda n, itself ~1e-6 sigma, by ~1e-13
// sigma, while g and every position and momentum update stay in float64.
__device__ __forceinline__ void surf_grad_f(const SysDev& S, float dx, float dy, float dz, float& nx, float& ny,
                                            float& nz) {
  switch (S.kind) {
    case kPlane: nx = S.p_f[0]; ny = S.p_f[1]; nz = S.p_f[2]; break;
    case kSphere: nx = 2.f * dx; ny = 2.f * dy; nz = 2.f * dz; break;
    case kEllipsoid:
      nx = 2.f * dx * S.inv_a2_f[0]; ny = 2.f * dy * S.inv_a2_f[1]; nz = 2.f * dz * S.inv_a2_f[2];
      break;
    case kTorus: {
      const float rho = sqrtf(fmaf(dx, dx, dy * dy));
      const float q = 2.f * (rho - S.p_f[0]) / rho;
      nx = q * dx; ny = q * dy; nz = 2.f * dz;
      break;
    }
    case kBump: {
      if (S.periodic[0]) dx -= S.box_len_f[0] * rintf(dx / S.box_len_f[0]);
      if (S.periodic[1]) dy -= S.box_len_f[1] * rintf(dy / S.box_len_f[1]);
      const float w2 = S.p_f[1] * S.p_f[1];
      const float e = S.p_f[0] * expf(-fmaf(dx, dx, dy * dy) / (2.f * w2)) / w2;
      nx = e * dx; ny = e * dy; nz = 1.f;
      break;
    }
    case kCylinder:
      nx = S.axis == 0 ? 0.f : 2.f * dx; ny = S.axis == 1 ? 0.f : 2.f * dy; nz = S.axis == 2 ? 0.f : 2.f * dz;
      break;
    default: nx = ny = nz = 0.f;
  }
}

// Visiting order of the pair kernel: a counting sort of the particles by a
// spatial key -- the system index in the top bits, then the Morton code of
// the particle's cell (coordinates interleaved bit by bit, so consecutive
// keys are compact octree blocks) with its low bits dropped to fit 2^20 keys.
// The order inside a key is the atomic order: it only decides which thread
// takes which particle, never a result.
__device__ __forceinline__ uint32_t part1by2(uint32_t v) {  // spread 10 bits to every third bit
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

struct OrderKey {
  uint32_t coord_shift;  // cell coordinates >> this keep 10 bits
  uint32_t morton_drop;  // low Morton bits dropped
  uint32_t sys_shift;    // system index << this
};

__device__ __forceinline__ uint32_t order_key(const DevArrays& A, const OrderKey& K, int64_t i) {
  const uint32_t sid = meta_sys(A.meta[i]);
  const SysDev& S = A.sys[sid];
  int cx, cy, cz;
  cell_decode(S, A.cell[i], cx, cy, cz);
  const uint32_t mort = part1by2((uint32_t)cx >> K.coord_shift) | (part1by2((uint32_t)cy >> K.coord_shift) << 1) |
                        (part1by2((uint32_t)cz >> K.coord_shift) << 2);
  return (sid << K.sys_shift) | (mort >> K.morton_drop);
}

__global__ void k_order_hist(DevArrays A, DevArrays O, OrderKey K) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  A.rank[i] = atomicAdd(&O.count[order_key(A, K, i)], 1u);
}

__global__ void k_order_scatter(DevArrays A, DevArrays O, OrderKey K, uint32_t* order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  order[O.start[order_key(A, K, i)] + A.rank[i]] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// pair forces
// ---------------------------------------------------------------------------
template <typename R> struct RecT;
template <> struct RecT<float> {
  using T = float4;
  static __device__ __forceinline__ uint32_t bits(const float4& r) { return __float_as_uint(r.w); }
};
template <> struct RecT<double> {
  using T = double4_32a;
  static __device__ __forceinline__ uint32_t bits(const double4_32a& r) {
    return (uint32_t)__double_as_longlong(r.w);
  }
};

// Tables of the mixed path's pair terms from double-float displacements
// (lj_term_acc); not loaded on the float64 path.
struct PairAcc {
  float rc2m[kMaxTypes * kMaxTypes];  // screen bound r_c^2 (1 + 2^-18)
  DF rc2[kMaxTypes * kMaxTypes];
  DF s6x2[kMaxTypes * kMaxTypes];     // 2 sigma^6
  float c24[kMaxTypes * kMaxTypes], c4[kMaxTypes * kMaxTypes], s6[kMaxTypes * kMaxTypes];
};

template <typename R> struct PairTab {
  R eps[kMaxTypes * kMaxTypes], sig2[kMaxTypes * kMaxTypes], rc2[kMaxTypes * kMaxTypes],
      shift[kMaxTypes * kMaxTypes], lin[kMaxTypes * kMaxTypes], rc[kMaxTypes * kMaxTypes];
  PairAcc acc;
};

template <typename R> __device__ __forceinline__ void load_tab(PairTab<R>& t, const TypeTable* T);
template <> __device__ __forceinline__ void load_tab<float>(PairTab<float>& t, const TypeTable* T) {
  for (int q = threadIdx.x; q < kMaxTypes * kMaxTypes; q += blockDim.x) {
    const int a = q / kMaxTypes, b = q % kMaxTypes;
    t.eps[q] = T->eps_f[a][b];
    t.sig2[q] = T->sig2_f[a][b];
    t.rc2[q] = T->rc2_f[a][b];
    t.shift[q] = T->shift_f[a][b];
    t.lin[q] = T->lin_f[a][b];
    t.rc[q] = T->rc_f[a][b];
    t.acc.rc2m[q] = T->rc2m_f[a][b];
    t.acc.rc2[q] = T->rc2_df[a][b];
    t.acc.s6x2[q] = T->s6x2_df[a][b];
    t.acc.c24[q] = T->c24_f[a][b];
    t.acc.c4[q] = T->c4_f[a][b];
    t.acc.s6[q] = T->s6_f[a][b];
  }
}
template <> __device__ __forceinline__ void load_tab<double>(PairTab<double>& t, const TypeTable* T) {
  for (int q = threadIdx.x; q < kMaxTypes * kMaxTypes; q += blockDim.x) {
    const int a = q / kMaxTypes, b = q % kMaxTypes;
    t.eps[q] = T->eps[a][b];
    t.sig2[q] = T->sig2[a][b];
    t.rc2[q] = T->rc2[a][b];
    t.shift[q] = T->shift[a][b];
    t.lin[q] = T->lin[a][b];
    t.rc[q] = T->rc[a][b];
  }
}

template <typename R> __device__ __forceinline__ R rcp(R v);
template <> __device__ __forceinline__ float rcp<float>(float v) { return __frcp_rn(v); }
template <> __device__ __forceinline__ double rcp<double>(double v) { return 1.0 / v; }

template <typename R> __device__ __forceinline__ R rsq(R v);
template <> __device__ __forceinline__ float rsq<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsq<double>(double v) { return nr_rsqrt(v); }

// Lennard-Jones pair term inside the cutoff (r2 < r_c^2), phi(r) = 4 eps
// [(s/r)^12 - (s/r)^6]: the truncated-shifted V = phi(r) - phi(r_c) of Eq. S1
// and, where the table holds phi'(r_c) != 0, the linearly smoothed form of the
// energy-conservation study, V = phi(r) - phi(r_c) - (r - r_c) phi'(r_c), whose
// force -phi'(r) + phi'(r_c) vanishes at r_c. Adds the force on i (along the
// displacement d = x_i - x_j) and half the pair energy.
template <typename R>
__device__ __forceinline__ void lj_term(const PairTab<R>& tab, uint32_t qt, R r2, R ddx, R ddy, R ddz, R& fx,
                                        R& fy, R& fz, R& u) {
  const R inv_r2 = rcp<R>(r2);
  const R s2 = tab.sig2[qt] * inv_r2;
  const R s6 = s2 * s2 * s2;
  const R e = tab.eps[qt];
  R fr = (R)24 * e * s6 * ((R)2 * s6 - (R)1) * inv_r2;
  R v = (R)4 * e * s6 * (s6 - (R)1) - tab.shift[qt];
  const R lin = tab.lin[qt];
  if (lin != (R)0) {
    const R inv_r = rsq<R>(r2);
    fr += lin * inv_r;
    v -= (r2 * inv_r - tab.rc[qt]) * lin;
  }
  fx += fr * ddx; fy += fr * ddy; fz += fr * ddz;
  u += (R)0.5 * v;
}

// Mixed path: the pair term of a candidate that the float32 screen found
// near or inside the cutoff, from the records' high parts (offsets from the
// cell centre rounded to float32) and low parts (the rounding remainders).
// Per axis the displacement d = (o_i - o_j - shift) is formed exactly as a
// double-float: two error-free sums (two_sum) of the high parts and the
// shift, plus the difference of the low parts. r^2 is then a double-float by
// Ogita, Rump and Oishi's compensated dot product (Dot2: exact squares by
// two_prod, exact partial sums by two_sum, the cross terms 2 d_h d_l), the
// cutoff test compares it with r_c^2 held as a double-float, and r^6 is a
// double-float product. The Lennard-Jones factor of Eq. S1 is written as
//   f(r)/r = 24 eps s6 (2 s6 - 1) / r^2 = 24 eps sigma^6 (2 sigma^6 - r^6) / (r^6 r^6 r^2),
// with 2 sigma^6 - r^6 formed from the double-float r^6 (exact cancellation
// near the WCA cutoff) and 1/r^6, 1/r^2 from a float32 reciprocal corrected
// by the low part. Only float32 products of well-conditioned factors remain,
// so the pair force carries a few float32 roundings relative to itself,
// while a float32 r^2 (relative error 2^-24) would move it by up to 22 of
// them near contact (d ln f / d ln r = -22 at r = 1.03 sigma) and by up to
// 6e-6 eps/sigma absolute near the WCA cutoff.
__device__ __forceinline__ DF pair_disp(float a, float b, float sh, float dl) {
  const DF s1 = df_two_sum(a, -b);
  const DF s2 = df_two_sum(s1.h, -sh);
  return {s2.h, __fadd_rn(__fadd_rn(s1.l, s2.l), dl)};
}

// One accurate pair term: the factor fr = f(r)/r, the displacement d and the
// pair energy v; false when r >= r_c.
struct AccTerm {
  float fr, v;
  DF dx, dy, dz;
};

__device__ __forceinline__ bool acc_pair(const PairTab<float>& tab, uint32_t qt, const float4& ri, const float4& li,
                                         const float4& rj, const float4& lj, float shx, float shy, float shz,
                                         AccTerm& t) {
  t.dx = pair_disp(ri.x, rj.x, shx, __fsub_rn(li.x, lj.x));
  t.dy = pair_disp(ri.y, rj.y, shy, __fsub_rn(li.y, lj.y));
  t.dz = pair_disp(ri.z, rj.z, shz, __fsub_rn(li.z, lj.z));
  const DF px = df_two_prod(t.dx.h, t.dx.h), py = df_two_prod(t.dy.h, t.dy.h), pz = df_two_prod(t.dz.h, t.dz.h);
  const DF s1 = df_two_sum(px.h, py.h);
  const DF s2 = df_two_sum(s1.h, pz.h);
  float lo = __fadd_rn(__fadd_rn(__fadd_rn(px.l, py.l), pz.l), __fadd_rn(s1.l, s2.l));
  lo = __fmaf_rn(2.f * t.dx.h, t.dx.l, lo);
  lo = __fmaf_rn(2.f * t.dy.h, t.dy.l, lo);
  lo = __fmaf_rn(2.f * t.dz.h, t.dz.l, lo);
  const DF r2 = df_fast_sum(s2.h, lo);
  const DF rc2 = tab.acc.rc2[qt];
  if (!(__fadd_rn(__fsub_rn(r2.h, rc2.h), __fsub_rn(r2.l, rc2.l)) < 0.f)) return false;  // r >= r_c
  const float iR0 = __frcp_rn(r2.h);
  const float iR = __fmaf_rn(-__fmul_rn(r2.l, iR0), iR0, iR0);  // 1 / r^2
  DF r4 = df_two_prod(r2.h, r2.h);
  r4.l = __fmaf_rn(2.f * r2.h, r2.l, r4.l);
  DF r6 = df_two_prod(r4.h, r2.h);
  r6.l = __fmaf_rn(r4.h, r2.l, __fmaf_rn(r4.l, r2.h, r6.l));
  const DF s = tab.acc.s6x2[qt];
  const float num = __fadd_rn(__fsub_rn(s.h, r6.h), __fsub_rn(s.l, r6.l));  // 2 sigma^6 - r^6
  const float iq0 = __frcp_rn(r6.h);
  const float iq = __fmaf_rn(-__fmul_rn(r6.l, iq0), iq0, iq0);  // 1 / r^6
  t.fr = tab.acc.c24[qt] * num * (iq * iq) * iR;
  const float s6 = tab.acc.s6[qt] * iq;
  t.v = tab.acc.c4[qt] * iq * (s6 - 1.f) - tab.shift[qt];
  const float lin = tab.lin[qt];
  if (lin != 0.f) {
    const float ir = rsqrtf(r2.h);
    t.fr += lin * ir;
    t.v -= (r2.h * ir - tab.rc[qt]) * lin;
  }
  return true;
}

// f += fr d (low part first), u += v / 2
__device__ __forceinline__ void acc_add(float fr, DF dx, DF dy, DF dz, float v, float& fx, float& fy, float& fz,
                                        float& u) {
  fx = __fmaf_rn(fr, dx.h, __fmaf_rn(fr, dx.l, fx));
  fy = __fmaf_rn(fr, dy.h, __fmaf_rn(fr, dy.l, fy));
  fz = __fmaf_rn(fr, dz.h, __fmaf_rn(fr, dz.l, fz));
  u += 0.5f * v;
}

__device__ __forceinline__ void lj_term_acc(const PairTab<float>& tab, uint32_t qt, const float4& ri,
                                            const float4& li, const float4& rj, const float4& lj, float shx,
                                            float shy, float shz, float& fx, float& fy, float& fz, float& u) {
  AccTerm t;
  if (acc_pair(tab, qt, ri, li, rj, lj, shx, shy, shz, t)) acc_add(t.fr, t.dx, t.dy, t.dz, t.v, fx, fy, fz, u);
}

// One candidate pair: float64 path as lj_term; mixed path a float32 screen on
// the records' high parts (r^2 < r_c^2 (1 + 2^-18); the screen's own error is
// below 2e-6 relative) and lj_term_acc for what passes, with the low part of
// the candidate's record loaded only then.
template <typename R>
__device__ __forceinline__ void pair_term(const PairTab<R>& tab, uint32_t qt, const typename RecT<R>::T& ri,
                                          const float4& li, const typename RecT<R>::T& rj,
                                          const float4* __restrict__ lo, uint32_t t, R shx, R shy, R shz, R& fx,
                                          R& fy, R& fz, R& u) {
  const R ddx = ri.x - rj.x - shx, ddy = ri.y - rj.y - shy, ddz = ri.z - rj.z - shz;
  const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
  if constexpr (sizeof(R) == 4) {
    if (r2 < tab.acc.rc2m[qt]) lj_term_acc(tab, qt, ri, li, rj, lo[t], shx, shy, shz, fx, fy, fz, u);
  } else {
    if (r2 < tab.rc2[qt]) lj_term<R>(tab, qt, r2, ddx, ddy, ddz, fx, fy, fz, u);
  }
}

template <typename R> __device__ __forceinline__ float4 rec_lo_at(const float4* lo, uint32_t s) {
  if constexpr (sizeof(R) == 4) return lo[s];
  return make_float4(0.f, 0.f, 0.f, 0.f);
}

// pair_term with the candidate's low part already loaded (lj; unused on the
// float64 path)
template <typename R>
__device__ __forceinline__ void pair_term_v(const PairTab<R>& tab, uint32_t qt, const typename RecT<R>::T& ri,
                                            const float4& li, const typename RecT<R>::T& rj, const float4& lj,
                                            R shx, R shy, R shz, R& fx, R& fy, R& fz, R& u) {
  const R ddx = ri.x - rj.x - shx, ddy = ri.y - rj.y - shy, ddz = ri.z - rj.z - shz;
  const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
  if constexpr (sizeof(R) == 4) {
    if (r2 < tab.acc.rc2m[qt]) lj_term_acc(tab, qt, ri, li, rj, lj, shx, shy, shz, fx, fy, fz, u);
  } else {
    if (r2 < tab.rc2[qt]) lj_term<R>(tab, qt, r2, ddx, ddy, ddz, fx, fy, fz, u);
  }
}

#ifndef SURFMD_NL_BATCH
#define SURFMD_NL_BATCH 2
#endif
constexpr int kNlBatch = SURFMD_NL_BATCH;  // list entries whose loads are in flight together

template <typename R> __device__ __forceinline__ void store_f(void* f, uint32_t i, R fx, R fy, R fz, R u);
template <> __device__ __forceinline__ void store_f<float>(void* f, uint32_t i, float fx, float fy, float fz,
                                                           float u) {
  reinterpret_cast<float4*>(f)[i] = make_float4(fx, fy, fz, u);
}
template <> __device__ __forceinline__ void store_f<double>(void* f, uint32_t i, double fx, double fy,
                                                            double fz, double u) {
  reinterpret_cast<double4_32a*>(f)[i] = make_double4_32a(fx, fy, fz, u);
}

// Minimum-image difference a - b of two positions of one system.
__device__ __forceinline__ void min_image_diff(const SysDev& S, const double* a, const double* b, double d[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d[k] = a[k] - b[k];
    if (S.periodic[k]) d[k] = wrap_min_image(d[k], S.box_len[k]);
  }
}

// Bend angle of three beads (SI S3.2): u = x_a - x_m, w = x_b - x_m,
// theta = atan2(|u x w|, u.w) (the angle at the middle bead, pi for a
// straight chain), V = k (theta - theta0)^2. With c = cos theta, s = sin
// theta and dV = 2k (theta - theta0), the force on a is (dV/s)(w/(|u||w|) -
// c u/|u|^2), on b the same with u and w exchanged, on m minus their sum
// (zero bracket at s = 0). `which` selects the bead (0 a, 1 m, 2 b); returns V.
__device__ __forceinline__ double bend_term(const SysDev& S, const double* xa, const double* xm, const double* xb,
                                            int which, double f[3]) {
  double u[3], w[3];
  min_image_diff(S, xa, xm, u);
  min_image_diff(S, xb, xm, w);
  const double uu = fma(u[0], u[0], fma(u[1], u[1], u[2] * u[2]));
  const double ww = fma(w[0], w[0], fma(w[1], w[1], w[2] * w[2]));
  const double uw = fma(u[0], w[0], fma(u[1], w[1], u[2] * w[2]));
  const double c0 = u[1] * w[2] - u[2] * w[1], c1 = u[2] * w[0] - u[0] * w[2], c2 = u[0] * w[1] - u[1] * w[0];
  const double sn = sqrt(fma(c0, c0, fma(c1, c1, c2 * c2)));
  const double theta = atan2(sn, uw);
  const double norm = sqrt(uu * ww);
  const double c = uw / norm, sth = sn / norm;
  const double dth = theta - S.angle_theta0;
  const double ratio = sth > 0.0 ? 2.0 * S.angle_k * dth / sth : 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double fa = ratio * (w[k] / norm - c * u[k] / uu);
    const double fb = ratio * (u[k] / norm - c * w[k] / ww);
    f[k] = which == 0 ? fa : (which == 2 ? fb : -(fa + fb));
  }
  return S.angle_k * dth * dth;
}

// The bend term on the mixed path. Float64 forms what cancels: u, w, the
// cross product C = u x w, u.w, |C| and the two arguments of
// dth = atan2(sin(theta - theta0), cos(theta - theta0)) (both scaled by
// |u||w|), so dth keeps float32's relative precision even near theta0 and near
// a straight chain. Float32 does the rest, with the brackets written without
// cancellation: w - (u.w / |u|^2) u = (C x u) / |u|^2 and
// u - (u.w / |w|^2) w = (w x C) / |w|^2.
__device__ __forceinline__ float bend_term_f(const SysDev& S, const double* xa, const double* xm, const double* xb,
                                             int which, float f[3]) {
  double u[3], w[3];
  min_image_diff(S, xa, xm, u);
  min_image_diff(S, xb, xm, w);
  const double C[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  const double uw = fma(u[0], w[0], fma(u[1], w[1], u[2] * w[2]));
  const double CC = fma(C[0], C[0], fma(C[1], C[1], C[2] * C[2]));
  const double sn = CC > 0.0 ? CC * nr_rsqrt(CC) : 0.0;  // |u||w| sin(theta)
  const float dth = atan2f(d2f_rn(fma(sn, S.angle_cos0, -uw * S.angle_sin0)),
                           d2f_rn(fma(uw, S.angle_cos0, sn * S.angle_sin0)));  // theta - theta0
  const float uf[3] = {d2f_rn(u[0]), d2f_rn(u[1]), d2f_rn(u[2])};
  const float wf[3] = {d2f_rn(w[0]), d2f_rn(w[1]), d2f_rn(w[2])};
  const float Cf[3] = {d2f_rn(C[0]), d2f_rn(C[1]), d2f_rn(C[2])};
  const float uu = fmaf(uf[0], uf[0], fmaf(uf[1], uf[1], uf[2] * uf[2]));
  const float ww = fmaf(wf[0], wf[0], fmaf(wf[1], wf[1], wf[2] * wf[2]));
  const float inv_norm = rsqrtf(uu * ww);
  const float sth = d2f_rn(sn) * inv_norm;
  const float k = (float)S.angle_k;
  const float ratio = sth > 0.f ? __fdividef(2.f * k * dth, sth) : 0.f;
  const float ga = __fdividef(ratio * inv_norm, uu), gb = __fdividef(ratio * inv_norm, ww);
  const float fa[3] = {ga * (Cf[1] * uf[2] - Cf[2] * uf[1]), ga * (Cf[2] * uf[0] - Cf[0] * uf[2]),
                       ga * (Cf[0] * uf[1] - Cf[1] * uf[0])};
  const float fb[3] = {gb * (wf[1] * Cf[2] - wf[2] * Cf[1]), gb * (wf[2] * Cf[0] - wf[0] * Cf[2]),
                       gb * (wf[0] * Cf[1] - wf[1] * Cf[0])};
#pragma unroll
  for (int q = 0; q < 3; ++q) f[q] = which == 0 ? fa[q] : (which == 2 ? fb[q] : -(fa[q] + fb[q]));
  return k * dth * dth;
}

// Bend angles of particle `tag` (float64 on the float64 path, float32 after
// float64 bond vectors on the mixed path): the force on it from every angle
// of three consecutive beads of its chain that contains it, and its energy
// share (a third of each angle). Kept out of the pair kernels (its registers
// would lower their occupancy): k_bend and a phase of the resident engine add
// it to the particle's force after the pair kernel.
template <typename R>
__device__ __forceinline__ void bend_on(const DevArrays& A, const SysDev& S, int64_t tag, R f[3], R& v) {
  const int64_t n = A.n;
  const int64_t pid = tag - S.first;
  const int64_t B = S.bpm;
  f[0] = f[1] = f[2] = (R)0;
  v = (R)0;
  for (int64_t mid = pid - 1; mid <= pid + 1; ++mid) {  // middle bead of each angle containing the particle
    if (mid < 1 || mid + 1 >= S.n || mid % B == 0 || mid % B == B - 1) continue;
    const int64_t gm = S.first + mid;
    const double xa[3] = {A.x[gm - 1], A.x[n + gm - 1], A.x[2 * n + gm - 1]};
    const double xm[3] = {A.x[gm], A.x[n + gm], A.x[2 * n + gm]};
    const double xb[3] = {A.x[gm + 1], A.x[n + gm + 1], A.x[2 * n + gm + 1]};
    R fa[3];
    if constexpr (sizeof(R) == 4) v += bend_term_f(S, xa, xm, xb, (int)(pid - mid + 1), fa) * (1.f / 3.f);
    else v += bend_term(S, xa, xm, xb, (int)(pid - mid + 1), fa) / 3.0;
    f[0] += fa[0]; f[1] += fa[1]; f[2] += fa[2];
  }
}

__device__ __forceinline__ bool has_bends(const SysDev& S) { return S.bpm > 2 && S.angle_k != 0.0; }

// Bonded and wall terms of particle `tag`: bonds V = k (r - r0)^2 (no factor
// 1/2) to the chain neighbours, r0 from the bead types when bond_mix is set,
// and the wall V_w (two z planes, or a sphere about wall_center) on
// unconstrained particles. The particle's energy share is half of each bond
// and all of its wall term. The float64 path works in float64 throughout.
// The mixed path forms in float64 only what cancels: the displacement, r^2
// and r^2 - r0^2 (the stretch r - r0 is small against r), the wall distance,
// or r^2 - R_w^2 for the spherical wall; then r - r0 = (r^2 - r0^2) / (r + r0)
// and the rest in float32, where the rounding of r enters denominators only.
__device__ __forceinline__ void bonded_terms_f(const DevArrays& A, const SysDev& S, uint32_t tag, uint32_t m,
                                               bool bonds, bool walls, float& fx, float& fy, float& fz,
                                               float& u) {
  const int64_t n = A.n;
  const double xi[3] = {A.x[tag], A.x[n + tag], A.x[2 * n + tag]};
  float bx = 0.f, by = 0.f, bz = 0.f, bu = 0.f;
  if (bonds && S.bpm > 1) {
    const int64_t pid = (int64_t)tag - S.first;
    const int64_t B = S.bpm;
    const float k = (float)S.bond_k;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      int64_t j;
      if (side == 0) {
        if (pid % B == 0) continue;
        j = (int64_t)tag - 1;
      } else {
        if (pid % B == B - 1 || pid + 1 >= S.n) continue;
        j = (int64_t)tag + 1;
      }
      const double xj[3] = {A.x[j], A.x[n + j], A.x[2 * n + j]};
      double d[3];
      min_image_diff(S, xi, xj, d);
      const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
      const double r0 = S.bond_mix ? A.types->bond_r0_mix[meta_type(m)][meta_type(A.meta[j])] : S.bond_r0;
      const float q = d2f_rn(fma(-r0, r0, r2));  // r^2 - r0^2
      const float r2f = d2f_rn(r2);
      const float ir = rsqrtf(r2f);
      const float dr = __fdividef(q, fmaf(r2f, ir, (float)r0));  // r - r0
      const float fo = -2.f * k * dr * ir;
      bx = fmaf(fo, d2f_rn(d[0]), bx);
      by = fmaf(fo, d2f_rn(d[1]), by);
      bz = fmaf(fo, d2f_rn(d[2]), bz);
      bu = fmaf(0.5f * k * dr, dr, bu);
    }
  }
  if (walls && S.wall && !meta_con(m)) {
    const float eps = (float)S.wall_eps, sig2 = (float)(S.wall_sigma * S.wall_sigma);
    if (S.wall_kind == 1) {
      const double d0 = xi[0] - S.wall_center[0], d1 = xi[1] - S.wall_center[1], d2 = xi[2] - S.wall_center[2];
      const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
      const float q = d2f_rn(fma(-S.wall_radius, S.wall_radius, r2));  // r^2 - R_w^2
      const float r2f = d2f_rn(r2);
      const float ir = rsqrtf(r2f);
      const float h = __fdividef(q, fmaf(r2f, ir, (float)S.wall_radius));  // r - R_w
      if (!(h > 0.f)) {
        flag(A.status, kFlagOutOfGrid);
      } else if (h < (float)S.wall_rc) {
        const float ih = __fdividef(1.f, h);
        const float s2 = sig2 * ih * ih;
        const float s6 = s2 * s2 * s2;
        const float fr = 24.f * eps * (2.f * s6 * s6 - s6) * ih * ir;
        bx = fmaf(fr, d2f_rn(d0), bx);
        by = fmaf(fr, d2f_rn(d1), by);
        bz = fmaf(fr, d2f_rn(d2), bz);
        bu += 4.f * eps * (s6 * s6 - s6 + 0.25f);
      }
    } else {
      const double dist[2] = {xi[2] - S.wall_lo, S.wall_hi - xi[2]};
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        if (!(dist[w] > 0.0)) {
          flag(A.status, kFlagOutOfGrid);
          continue;
        }
        if (dist[w] >= S.wall_rc) continue;
        const float ir = __fdividef(1.f, d2f_rn(dist[w]));
        const float s2 = sig2 * ir * ir;
        const float s6 = s2 * s2 * s2;
        const float fr = 24.f * eps * (2.f * s6 * s6 - s6) * ir;
        bz += (w == 0) ? fr : -fr;
        bu += 4.f * eps * (s6 * s6 - s6 + 0.25f);
      }
    }
  }
  fx += bx; fy += by; fz += bz; u += bu;
}

template <typename R>
__device__ __forceinline__ void bonded_terms(const DevArrays& A, const SysDev& S, uint32_t tag, uint32_t m,
                                             bool bonds, bool walls, R& fx, R& fy, R& fz, R& u) {
  if constexpr (sizeof(R) == 4) {
    bonded_terms_f(A, S, tag, m, bonds, walls, fx, fy, fz, u);
    return;
  }
  const int64_t n = A.n;
  const double xi[3] = {A.x[tag], A.x[n + tag], A.x[2 * n + tag]};
  double bx = 0.0, by = 0.0, bz = 0.0, bu = 0.0;
  if (bonds && S.bpm > 1) {
    const int64_t pid = (int64_t)tag - S.first;
    const int64_t B = S.bpm;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      int64_t j;
      if (side == 0) {
        if (pid % B == 0) continue;
        j = (int64_t)tag - 1;
      } else {
        if (pid % B == B - 1 || pid + 1 >= S.n) continue;
        j = (int64_t)tag + 1;
      }
      const double xj[3] = {A.x[j], A.x[n + j], A.x[2 * n + j]};
      double d[3];
      min_image_diff(S, xi, xj, d);
      const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
      const double ir = nr_rsqrt(r2);
      const double r0 = S.bond_mix ? A.types->bond_r0_mix[meta_type(m)][meta_type(A.meta[j])] : S.bond_r0;
      const double dr = fma(r2, ir, -r0);  // r - r0
      const double fo = -2.0 * S.bond_k * dr * ir;
      bx = fma(fo, d[0], bx); by = fma(fo, d[1], by); bz = fma(fo, d[2], bz);
      bu = fma(0.5 * S.bond_k * dr, dr, bu);
    }
  }
  if (walls && S.wall && !meta_con(m)) {
    if (S.wall_kind == 1) {
      const double d0 = xi[0] - S.wall_center[0], d1 = xi[1] - S.wall_center[1], d2 = xi[2] - S.wall_center[2];
      const double r = sqrt(fma(d0, d0, fma(d1, d1, d2 * d2)));
      const double h = r - S.wall_radius;
      if (!(h > 0.0)) {
        flag(A.status, kFlagOutOfGrid);
      } else if (h < S.wall_rc) {
        const double ih = nr_rcp(h);
        const double s2 = S.wall_sigma * S.wall_sigma * ih * ih;
        const double s6 = s2 * s2 * s2;
        const double fr = 24.0 * S.wall_eps * (2.0 * s6 * s6 - s6) * ih / r;
        bx = fma(fr, d0, bx); by = fma(fr, d1, by); bz = fma(fr, d2, bz);
        bu += 4.0 * S.wall_eps * (s6 * s6 - s6 + 0.25);
      }
    } else {
      const double dist[2] = {xi[2] - S.wall_lo, S.wall_hi - xi[2]};
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const double r = dist[w];
        if (!(r > 0.0)) {
          flag(A.status, kFlagOutOfGrid);
          continue;
        }
        if (r >= S.wall_rc) continue;
        const double ir = nr_rcp(r);
        const double s2 = S.wall_sigma * S.wall_sigma * ir * ir;
        const double s6 = s2 * s2 * s2;
        const double fr = 24.0 * S.wall_eps * (2.0 * s6 * s6 - s6) * ir;
        bz += (w == 0) ? fr : -fr;
        bu += 4.0 * S.wall_eps * (s6 * s6 - s6 + 0.25);
      }
    }
  }
  fx += (R)bx; fy += (R)by; fz += (R)bz; u += (R)bu;
}

// The cell list as the pair code reads it: slot -> particle, cell and record,
// bucket -> first slot, cell -> bucket. GlobalCells is the handle's list in
// global memory; the resident engine keeps one system's list in shared memory.
template <typename R> struct GlobalCells {
  using Rec = typename RecT<R>::T;
  const Rec* __restrict__ rec_;
  const float4* __restrict__ lo_;
  const uint32_t* __restrict__ scell_;
  const uint32_t* __restrict__ start_;
  const uint32_t* __restrict__ stag_;
  int hashed, log_t;
  __device__ __forceinline__ explicit GlobalCells(const DevArrays& A)
      : rec_(reinterpret_cast<const Rec*>(A.rec)), lo_(A.rec_lo), scell_(A.scell), start_(A.start), stag_(A.stag),
        hashed(A.hashed), log_t(A.log_t) {}
  __device__ __forceinline__ const float4* lo() const { return lo_; }
  __device__ __forceinline__ uint32_t tag(uint32_t s) const { return stag_[s]; }
  __device__ __forceinline__ uint32_t scell(uint32_t t) const { return scell_[t]; }
  __device__ __forceinline__ Rec rec(uint32_t t) const { return rec_[t]; }
  __device__ __forceinline__ uint32_t start(uint32_t b) const { return start_[b]; }
  __device__ __forceinline__ uint32_t bucket(uint32_t cell) const { return bucket_of(cell, hashed, log_t); }
};

template <typename R, bool BONDS, bool WALLS, bool EXCL, class Cells>
__device__ __forceinline__ uint32_t pair_slot(const DevArrays& A, const Cells& C, const PairTab<R>& tab, uint32_t s,
                                              R& fx, R& fy, R& fz, R& u) {
  using Rec = typename RecT<R>::T;
  const uint32_t tag = C.tag(s);
  const uint32_t cell = C.scell(s);
  const Rec ri = C.rec(s);
  const float4 li = rec_lo_at<R>(C.lo(), s);
  const uint32_t bi = RecT<R>::bits(ri);
  const uint32_t ti = bi & 7u, moli = bi >> 3;
  const uint32_t m = A.meta[tag];
  const uint32_t sid = meta_sys(m);
  const SysDev& S = A.sys[sid];
  int c[3];
  cell_decode(S, cell, c[0], c[1], c[2]);
  // stencil shift: the cell edge in R (float edges are exact on open axes)
  const R csx = sizeof(R) == 4 ? (R)S.cs_f[0] : (R)S.cs[0];
  const R csy = sizeof(R) == 4 ? (R)S.cs_f[1] : (R)S.cs[1];
  const R csz = sizeof(R) == 4 ? (R)S.cs_f[2] : (R)S.cs[2];
  // tangent-slab pruning
  bool prune = S.slab > 0.f && meta_con(m) && A.sys_free[sid] == 0;
  float nhx = 0.f, nhy = 0.f, nhz = 0.f, reach = 0.f, on = 0.f;
  if (prune) {
    const float ox = (float)ri.x, oy = (float)ri.y, oz = (float)ri.z;
    const float rx = S.grid_lo_f[0] + ((float)c[0] + 0.5f) * S.cs_f[0] + ox - S.c_f[0];
    const float ry = S.grid_lo_f[1] + ((float)c[1] + 0.5f) * S.cs_f[1] + oy - S.c_f[1];
    const float rz = S.grid_lo_f[2] + ((float)c[2] + 0.5f) * S.cs_f[2] + oz - S.c_f[2];
    surf_grad_f(S, rx, ry, rz, nhx, nhy, nhz);
    const float nn = fmaf(nhx, nhx, fmaf(nhy, nhy, nhz * nhz));
    if (nn > 0.f) {
      const float inv = rsqrtf(nn);
      nhx *= inv; nhy *= inv; nhz *= inv;
      reach = 0.5f * (S.cs_f[0] * fabsf(nhx) + S.cs_f[1] * fabsf(nhy) + S.cs_f[2] * fabsf(nhz)) + S.slab;
      on = nhx * ox + nhy * oy + nhz * oz;
    } else {
      prune = false;
    }
  }
  fx = 0; fy = 0; fz = 0; u = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int z = c[2] + dz;
    if (z < 0 || z >= S.nc[2]) {
      if (!S.periodic[2]) continue;
      z = (z + S.nc[2]) % S.nc[2];
    }
    for (int dy = -1; dy <= 1; ++dy) {
      int y = c[1] + dy;
      if (y < 0 || y >= S.nc[1]) {
        if (!S.periodic[1]) continue;
        y = (y + S.nc[1]) % S.nc[1];
      }
      uint32_t nb[3], t0[3], t1[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int dx = q - 1;
        t0[q] = 0u;
        t1[q] = 0u;
        nb[q] = 0u;
        int x = c[0] + dx;
        if (x < 0 || x >= S.nc[0]) {
          if (!S.periodic[0]) continue;
          x = (x + S.nc[0]) % S.nc[0];
        }
        if (prune) {
          const float dist = nhx * (float)dx * S.cs_f[0] + nhy * (float)dy * S.cs_f[1] +
                             nhz * (float)dz * S.cs_f[2] - on;
          if (fabsf(dist) > reach) continue;
        }
        nb[q] = cell_id(S, x, y, z);
        const uint32_t b = C.bucket(nb[q]);
        t0[q] = C.start(b);
        t1[q] = C.start(b + 1);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const R shx = (R)(q - 1) * csx, shy = (R)dy * csy, shz = (R)dz * csz;
        for (uint32_t t = t0[q]; t < t1[q]; ++t) {
          const Rec rj = C.rec(t);
          const uint32_t cj = A.rec_cell ? RecT<R>::bits(rj) >> 3 : C.scell(t);
          if (cj != nb[q] || t == s) continue;
          const uint32_t bj = RecT<R>::bits(rj);
          if (EXCL && (bj >> 3) == moli) continue;
          const uint32_t qt = ti * kMaxTypes + (bj & 7u);
          pair_term<R>(tab, qt, ri, li, rj, C.lo(), t, shx, shy, shz, fx, fy, fz, u);
        }
      }
    }
  }
  if (BONDS || WALLS) bonded_terms<R>(A, S, tag, m, BONDS, WALLS, fx, fy, fz, u);
  return tag;
}

template <typename R, bool BONDS, bool WALLS, bool EXCL>
__global__ void __launch_bounds__(256) k_pair_row(DevArrays A) {
  __shared__ PairTab<R> tab;
  load_tab<R>(tab, A.types);
  __syncthreads();
  const uint32_t t_id = blockIdx.x * blockDim.x + threadIdx.x;
  if (t_id >= (uint32_t)A.n) return;
  // with a visiting order, neighbouring threads take spatially neighbouring
  // particles, whose stencils share cache lines; the particle's own slot
  // follows from the slot map (the arithmetic per particle is unchanged)
  const uint32_t s = A.order ? A.slot_of[A.order[t_id]] : t_id;
  R fx, fy, fz, u;
  const uint32_t tag = pair_slot<R, BONDS, WALLS, EXCL>(A, GlobalCells<R>(A), tab, s, fx, fy, fz, u);
  store_f<R>(A.f, tag, fx, fy, fz, u);
}

// ---------------------------------------------------------------------------
// Verlet neighbour list. k_nl_build (one thread per sorted slot, only when
// the rebuild flag is up) lists every pair within r_c + skin of the fresh
// cell list: entry = neighbour slot << 5 | stencil cell k (k = 9(dz+1) +
// 3(dy+1) + dx+1, the shift of the neighbour's cell), in stencil order, no
// self pair, no same-molecule pair; it also keeps the records and the
// positions of the build. k_pair_nl walks the list with the records the
// integrator moved in place, with the row kernel's arithmetic (the cell
// edge is at least r_c + skin, so a particle within skin / 2 of its build
// position is still within r_c + skin of any partner it had).
// ---------------------------------------------------------------------------
#ifndef SURFMD_NL_BUILD_BATCH
#define SURFMD_NL_BUILD_BATCH 2
#endif
constexpr int kNlBuildBatch = SURFMD_NL_BUILD_BATCH;

template <typename R, bool EXCL>
__device__ __forceinline__ uint32_t nl_build_one(const DevArrays& A, const PairTab<R>& tab, uint32_t s) {
  using Rec = typename RecT<R>::T;
  const GlobalCells<R> C(A);
  const int64_t n = A.n;
  const uint32_t tag = C.tag(s);
  const uint32_t cell = C.scell(s);
  const Rec ri = C.rec(s);
  const uint32_t bi = RecT<R>::bits(ri);
  const uint32_t ti = bi & 7u, moli = bi >> 3;
  const SysDev& S = A.sys[meta_sys(A.meta[tag])];
  int c[3];
  cell_decode(S, cell, c[0], c[1], c[2]);
  const R csx = sizeof(R) == 4 ? (R)S.cs_f[0] : (R)S.cs[0];
  const R csy = sizeof(R) == 4 ? (R)S.cs_f[1] : (R)S.cs[1];
  const R csz = sizeof(R) == 4 ? (R)S.cs_f[2] : (R)S.cs[2];
  const R skin = (R)A.nl_skin;
  const uint32_t cap = (uint32_t)A.nl_max;
  uint32_t cnt = 0;
  // the candidates of a run of len cells with consecutive ids and consecutive
  // buckets (x = x0 .. x0 + len - 1 of one row) are one contiguous range of
  // slots, the cells' particles one after another: the same candidates in
  // the same order as cell by cell, with one pair of bucket bounds per run
  // (the candidates' records are loaded kNlBuildBatch at a time, so their
  // loads are in flight together; they are tested in slot order)
  auto walk = [&](uint32_t cell0, uint32_t b0, uint32_t len, int dx0, int dy, int dz) {
    const uint32_t t1 = C.start(b0 + len);
    const R shy = (R)dy * csy, shz = (R)dz * csz;
    for (uint32_t t0 = C.start(b0); t0 < t1; t0 += kNlBuildBatch) {
      Rec rb[kNlBuildBatch];
      uint32_t cb[kNlBuildBatch];
#pragma unroll
      for (int q = 0; q < kNlBuildBatch; ++q) {
        if (t0 + q < t1) {
          rb[q] = C.rec(t0 + q);
          cb[q] = A.rec_cell ? RecT<R>::bits(rb[q]) >> 3 : C.scell(t0 + q);
        }
      }
#pragma unroll
      for (int q = 0; q < kNlBuildBatch; ++q) {
        const uint32_t t = t0 + q;
        if (t >= t1) break;
        const Rec& rj = rb[q];
        const uint32_t k = cb[q] - cell0;  // which cell of the run (a hash collision: none)
        if (k >= len || t == s) continue;
        const uint32_t bj = RecT<R>::bits(rj);
        if (EXCL && (bj >> 3) == moli) continue;
        const uint32_t qt = ti * kMaxTypes + (bj & 7u);
        if (!(tab.rc2[qt] > (R)0)) continue;
        const int dx = dx0 + (int)k;
        const R ddx = ri.x - rj.x - (R)dx * csx, ddy = ri.y - rj.y - shy, ddz = ri.z - rj.z - shz;
        const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        const R rs = tab.rc[qt] + skin;
        if (r2 < rs * rs) {
          if (cnt < cap) A.nl[(int64_t)s * cap + cnt] = t << 5 | (uint32_t)(9 * (dz + 1) + 3 * (dy + 1) + dx + 1);
          ++cnt;
        }
      }
    }
  };
  for (int dz = -1; dz <= 1; ++dz) {
    int z = c[2] + dz;
    if (z < 0 || z >= S.nc[2]) {
      if (!S.periodic[2]) continue;
      z = (z + S.nc[2]) % S.nc[2];
    }
    for (int dy = -1; dy <= 1; ++dy) {
      int y = c[1] + dy;
      if (y < 0 || y >= S.nc[1]) {
        if (!S.periodic[1]) continue;
        y = (y + S.nc[1]) % S.nc[1];
      }
      // the row's three cells (dx = -1, 0, +1; the first and last may be
      // missing on an open axis or wrapped on a periodic one)
      int xm = c[0] - 1, xp = c[0] + 1;
      bool hm = true, hp = true;
      if (xm < 0) {
        hm = S.periodic[0] != 0;
        xm += S.nc[0];
      }
      if (xp >= S.nc[0]) {
        hp = S.periodic[0] != 0;
        xp -= S.nc[0];
      }
      const uint32_t cc = cell_id(S, c[0], y, z), bc = C.bucket(cc);
      const uint32_t cm = hm ? cell_id(S, xm, y, z) : 0u, bm = hm ? C.bucket(cm) : 0u;
      const uint32_t cp = hp ? cell_id(S, xp, y, z) : 0u, bp = hp ? C.bucket(cp) : 0u;
      const bool jm = hm && cc == cm + 1u && bc == bm + 1u;  // dx = -1 joins the centre's run
      const bool jp = hp && cp == cc + 1u && bp == bc + 1u;  // dx = +1 joins it
      // the row's runs in dx order: [-1 alone], the centre's run, [+1 alone]
#pragma unroll 1
      for (int r = (hm && !jm) ? 0 : 1; r <= ((hp && !jp) ? 2 : 1); ++r) {
        const uint32_t c0 = r == 0 ? cm : r == 2 ? cp : (jm ? cm : cc);
        const uint32_t b0 = r == 0 ? bm : r == 2 ? bp : (jm ? bm : bc);
        const uint32_t len = r == 1 ? 1u + (jm ? 1u : 0u) + (jp ? 1u : 0u) : 1u;
        const int dx0 = r == 0 ? -1 : r == 2 ? 1 : (jm ? -1 : 0);
        walk(c0, b0, len, dx0, dy, dz);
      }
    }
  }
  if (cnt > cap) flag(A.status, kFlagNlistFull);
  A.nl_cnt[s] = min(cnt, cap);
  reinterpret_cast<Rec*>(A.rec0)[tag] = ri;  // by particle: the integrator reads it in particle order
  if (sizeof(R) == 4) A.rec0_lo[tag] = A.rec_lo[s];
  A.xb[tag] = A.x[tag];
  A.xb[n + tag] = A.x[n + tag];
  A.xb[2 * n + tag] = A.x[2 * n + tag];
  return min(cnt, cap);
}

// Packs the lists of a warp's 32 consecutive slots s (group-aligned; lanes
// past the end pass valid = false) into their group's run of nl_pk: a prefix
// sum of the counts over the warp gives each slot's start, and each lane
// copies its own entries from the scratch it has just written.
__device__ __forceinline__ void nl_pack_warp(const DevArrays& A, uint32_t s, bool valid, uint32_t cnt) {
  const int lane = (int)(threadIdx.x & 31u);
  const uint32_t c = valid ? cnt : 0u;
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (!valid) return;
  const uint32_t pre = incl - c;
  const uint32_t cap = (uint32_t)A.nl_max;
  A.nl_off[s] = pre;
  const uint32_t* src = A.nl + (int64_t)s * cap;
  uint32_t* dst = A.nl_pk + (int64_t)(s & ~31u) * cap + pre;
  for (uint32_t k = 0; k < c; ++k) dst[k] = src[k];
}

template <typename R, bool EXCL>
__global__ void __launch_bounds__(256) k_nl_build(DevArrays A) {
  __shared__ PairTab<R> tab;
  if (*A.nl_dirty == 0u) return;  // uniform: nothing moved far enough
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.nl_builds += 1ull;
  load_tab<R>(tab, A.types);
  __syncthreads();
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;  // whole warps: blockDim is a multiple of 32
  const bool valid = s < (uint32_t)A.n;
  const uint32_t cnt = valid ? nl_build_one<R, EXCL>(A, tab, s) : 0u;
  nl_pack_warp(A, s, valid, cnt);
}

// ---------------------------------------------------------------------------
// Fused rebuild (Verlet-list step form): one cooperative launch per step that
// returns at once unless a particle has moved skin / 2 since the last build;
// then it runs the cell-list build (binning, exclusive scan of the bucket
// counters, scatter, canonical order and records) and the list build, with a
// grid barrier between phases, in place of five launches of which four would
// exit at once. Every CTA of a cooperative launch is resident, so the barrier
// cannot wait for a CTA that never runs; its wait is bounded all the same
// (spin_limit polls; on running out the CTA latches the timeout flag and the
// whole grid leaves, the host rebuilding the list before the next step).
// Each phase's per-item work is the separate kernels' own (bin_one,
// scatter_one, bucket_build_one, nl_build_one): the same list, bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(GridBar* b, uint32_t nblocks, uint32_t limit, uint32_t* status,
                                             int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* gen = &b->gen;
    const uint32_t g0 = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&b->count, 1u) == nblocks - 1) {  // last to arrive: release the others
      b->count = 0u;
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      uint32_t polls = 0;
      while (*gen == g0 && polls < limit) ++polls;
      if (*gen == g0) {
        ok = 0;
        atomicOr(status, kFlagTimeout);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

#ifndef SURFMD_REBUILD_THREADS
#define SURFMD_REBUILD_THREADS 256
#endif
constexpr int kRebuildThreads = SURFMD_REBUILD_THREADS;  // threads per CTA of the fused rebuild

template <typename R, bool EXCL>
__global__ void __launch_bounds__(kRebuildThreads) k_rebuild(DevArrays A) {
  __shared__ PairTab<R> tab;
  __shared__ uint32_t warp_tot[33];
  __shared__ int s_ok;
  __shared__ uint32_t s_pre;
  const uint32_t G = gridDim.x, tid = threadIdx.x, bd = blockDim.x;
  const bool lead = blockIdx.x == 0 && tid == 0;
  if (*A.nl_dirty == 0u) {  // uniform: nothing moved far enough; only the step advances
    if (lead) {
      if (A.noise_k) *A.noise_k = *A.step;  // the integrator has stored this step's normals
      *A.step += 1ull;
      *A.mode = 1;
    }
    return;
  }
  load_tab<R>(tab, A.types);
  const int64_t n = A.n;
  const int64_t stride = (int64_t)G * bd;
  const int64_t first = (int64_t)blockIdx.x * bd + tid;
  const uint32_t T = A.nbucket, lim = A.spin_limit;
  // 1. cell of every particle and its rank in the bucket counter
  for (int64_t i = first; i < n; i += stride) bin_one<R>(A, i);
  if (!grid_barrier(A.gbar, G, lim, A.status, &s_ok)) return;
  // 2. exclusive scan of the counters: each CTA a contiguous range, its sum,
  //    then (after the barrier) the sums of the CTAs before it as its prefix
  const uint32_t chunk = (T + G - 1) / G;
  const uint32_t b0 = min(blockIdx.x * chunk, T), b1 = min(b0 + chunk, T);
  uint32_t part = 0;
  for (uint32_t b = b0 + tid; b < b1; b += bd) part += A.count[b];
  uint32_t total;
  block_exclusive_scan(part, warp_tot, total);
  if (tid == 0) A.rb_sum[blockIdx.x] = total;
  if (!grid_barrier(A.gbar, G, lim, A.status, &s_ok)) return;
  part = 0;
  for (uint32_t j = tid; j < blockIdx.x; j += bd) part += A.rb_sum[j];
  block_exclusive_scan(part, warp_tot, total);
  if (tid == 0) s_pre = total;
  __syncthreads();
  uint32_t run = s_pre;
  for (uint32_t base = b0; base < b1; base += bd) {  // bd counters at a time, in order
    const uint32_t b = base + tid;
    const uint32_t v = b < b1 ? A.count[b] : 0u;
    const uint32_t ex = block_exclusive_scan(v, warp_tot, total);
    if (b < b1) {
      A.start[b] = run + ex;
      A.count[b] = 0u;
    }
    run += total;
    __syncthreads();  // every thread has read this round's totals before the next round writes them
  }
  if (!grid_barrier(A.gbar, G, lim, A.status, &s_ok)) return;
  // 3. particles to their slots (atomic order), 4. canonical order and records
  for (int64_t i = first; i < n; i += stride) scatter_one(A, i);
  if (!grid_barrier(A.gbar, G, lim, A.status, &s_ok)) return;
  for (int64_t s = first; s < n; s += stride) bucket_build_one<R>(A, s);
  if (!grid_barrier(A.gbar, G, lim, A.status, &s_ok)) return;
  // 5. the Verlet list of the new cell list, packed by whole warps of 32 consecutive slots
  for (int64_t w = first - (tid & 31u); w < n; w += stride) {
    const int64_t s = w + (tid & 31u);
    const bool valid = s < n;
    const uint32_t cnt = valid ? nl_build_one<R, EXCL>(A, tab, (uint32_t)s) : 0u;
    nl_pack_warp(A, (uint32_t)s, valid, cnt);
  }
  if (lead) {
    *A.nl_builds += 1ull;
    if (A.noise_k) *A.noise_k = *A.step;
    *A.step += 1ull;
    *A.mode = 1;
  }
}

// CTAs of the fused rebuild: at most what is resident at once on the device
// (a cooperative launch needs it), at most kRebuildMaxBlocks, no more than
// the particles need.
int rebuild_blocks(int precision, int excl, int64_t n) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return 0;
  cudaError_t e;
  if (precision == 0) {
    e = excl ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rebuild<double, true>, kRebuildThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rebuild<double, false>, kRebuildThreads, 0);
  } else {
    e = excl ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rebuild<float, true>, kRebuildThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rebuild<float, false>, kRebuildThreads, 0);
  }
  if (e != cudaSuccess || per_sm < 1) return 0;
  const int64_t want = std::max<int64_t>(1, (n + kRebuildThreads - 1) / kRebuildThreads);
  return (int)std::min<int64_t>({want, (int64_t)per_sm * sms, (int64_t)kRebuildMaxBlocks});
}

cudaError_t launch_rebuild(const DevArrays& A, int precision, int excl, int blocks, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kRebuildThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (precision == 0) {
    return excl ? cudaLaunchKernelEx(&cfg, k_rebuild<double, true>, A) : cudaLaunchKernelEx(&cfg, k_rebuild<double, false>, A);
  }
  return excl ? cudaLaunchKernelEx(&cfg, k_rebuild<float, true>, A) : cudaLaunchKernelEx(&cfg, k_rebuild<float, false>, A);
}

#ifndef SURFMD_PAIR_NL_MINB
#define SURFMD_PAIR_NL_MINB 1
#endif

template <typename R, bool BONDS, bool WALLS>
__global__ void __launch_bounds__(256, SURFMD_PAIR_NL_MINB) k_pair_nl(DevArrays A) {
  __shared__ PairTab<R> tab;
  load_tab<R>(tab, A.types);
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.nl_dirty = 0u;  // the previous step's rebuild is done
  __syncthreads();
  using Rec = typename RecT<R>::T;
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (uint32_t)A.n) return;
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(A.rec);
  const uint32_t tag = A.stag[s];
  const uint32_t m = A.meta[tag];
  const SysDev& S = A.sys[meta_sys(m)];
  const Rec ri = rec[s];
  const float4* __restrict__ lo = A.rec_lo;
  const float4 li = rec_lo_at<R>(lo, s);
  const uint32_t ti = RecT<R>::bits(ri) & 7u;
  const R csx = sizeof(R) == 4 ? (R)S.cs_f[0] : (R)S.cs[0];
  const R csy = sizeof(R) == 4 ? (R)S.cs_f[1] : (R)S.cs[1];
  const R csz = sizeof(R) == 4 ? (R)S.cs_f[2] : (R)S.cs[2];
  const uint32_t cnt = A.nl_cnt[s];
  const uint32_t* __restrict__ nl = A.nl_pk + (int64_t)(s & ~31u) * A.nl_max + A.nl_off[s];
  R fx = 0, fy = 0, fz = 0, u = 0;
  // batches of kNlBatch entries: the batch's entries, then its records (and,
  // mixed, their low parts) are all loaded before any term is evaluated, so
  // the gathers of a batch are in flight together; the terms are added in
  // list order, as one entry at a time would add them
  uint32_t k = 0;
  for (; k + kNlBatch <= cnt; k += kNlBatch) {
    uint32_t e[kNlBatch];
    Rec rj[kNlBatch];
    float4 lj[kNlBatch];
#pragma unroll
    for (int q = 0; q < kNlBatch; ++q) e[q] = nl[k + q];
#pragma unroll
    for (int q = 0; q < kNlBatch; ++q) {
      rj[q] = rec[e[q] >> 5];
      lj[q] = rec_lo_at<R>(lo, e[q] >> 5);
    }
#pragma unroll
    for (int q = 0; q < kNlBatch; ++q) {
      const uint32_t code = e[q] & 31u;
      const int dz = (int)(code / 9u) - 1, dy = (int)(code / 3u % 3u) - 1, dx = (int)(code % 3u) - 1;
      const uint32_t qt = ti * kMaxTypes + (RecT<R>::bits(rj[q]) & 7u);
      pair_term_v<R>(tab, qt, ri, li, rj[q], lj[q], (R)dx * csx, (R)dy * csy, (R)dz * csz, fx, fy, fz, u);
    }
  }
  for (; k < cnt; ++k) {
    const uint32_t e = nl[k];
    const uint32_t code = e & 31u;
    const Rec rj = rec[e >> 5];
    const int dz = (int)(code / 9u) - 1, dy = (int)(code / 3u % 3u) - 1, dx = (int)(code % 3u) - 1;
    const uint32_t qt = ti * kMaxTypes + (RecT<R>::bits(rj) & 7u);
    pair_term<R>(tab, qt, ri, li, rj, lo, e >> 5, (R)dx * csx, (R)dy * csy, (R)dz * csz, fx, fy, fz, u);
  }
  if (BONDS || WALLS) bonded_terms<R>(A, S, tag, m, BONDS, WALLS, fx, fy, fz, u);
  store_f<R>(A.f, tag, fx, fy, fz, u);
}

// Mixed path with the Verlet list, one warp per list_warp (8, 16 or 32)
// consecutive slots (fewer for long lists, so more warps share the work). The
// warp walks its particles' list entries as one flat sequence (particle by
// particle, each particle's entries in list order; its list is contiguous, so
// 32 consecutive positions are a few contiguous runs), kNlqGroup chunks of 32
// positions at a time: lane q takes positions c + q, c + 32 + q, ..., finds
// each one's particle by a binary search over the warp's prefix sums of the
// list lengths and loads the entries; the entries' records and low parts are
// then copied to shared memory with cp.async, all of the group's copies in
// flight together and no register held for them. The pairs are screened in
// float32 on the staged high parts; those that pass are queued (a ballot
// gives each its place, in the flat order) and evaluated 32 at a time on all
// lanes with the double-float arithmetic of lj_term_acc. A particle's queued
// pairs are consecutive, so after each evaluation the particle's lane adds its
// run of terms in order: every particle adds its terms in list order with the
// same arithmetic as k_pair_nl (the same bits), while no lane idles on a short
// list or on a pair that fails the screen.
constexpr int kQueueWarps = 8;
#ifndef SURFMD_NLQ_GROUP
#define SURFMD_NLQ_GROUP 3
#endif
#ifndef SURFMD_NLQ_MINB
#define SURFMD_NLQ_MINB 1
#endif
constexpr int kNlqGroup = SURFMD_NLQ_GROUP;
constexpr int kNlqStage = 32 * kNlqGroup;  // staged positions per warp

struct QueueWarp {
  float4 ri[32], li[32];  // the lanes' own records and low parts
  // staged pairs: the neighbour's record and low part; an evaluation
  // overwrites a staged pair with its term, (fr, dx.h, dy.h, dz.h) and
  // (dx.l, dy.l, dz.l, v)
  float4 sr[kNlqStage], sl[kNlqStage];
  float csx[32], csy[32], csz[32];  // the lanes' cell edges (their systems')
  uint8_t code[kNlqStage];          // staged pair: stencil cell of the neighbour
  uint8_t own[kNlqStage];           // staged pair: its particle (lane)
  uint8_t in[kNlqStage];            // staged pair: evaluated term is inside the cutoff
  uint8_t q[kNlqStage];             // queue: staged pairs that passed the screen, in order
  uint8_t run0[32], runn[32];       // per particle: first queue position and length of its run
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <bool BONDS, bool WALLS>
__global__ void __launch_bounds__(kQueueWarps * 32, SURFMD_NLQ_MINB) k_pair_nlq(DevArrays A) {
  __shared__ PairTab<float> tab;
  __shared__ QueueWarp qw_all[kQueueWarps];
  load_tab<float>(tab, A.types);
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.nl_dirty = 0u;  // the previous step's rebuild is done
  const int lane = (int)(threadIdx.x & 31u);
  QueueWarp& Q = qw_all[threadIdx.x >> 5];
  __syncthreads();
  // the warp's particles: list_warp (8, 16 or 32) consecutive slots, one per lane from lane 0
  const uint32_t P = (uint32_t)A.list_warp;
  const uint32_t s0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * P;  // the warp's first slot
  const uint32_t s = s0 + (uint32_t)lane;
  const bool valid = (uint32_t)lane < P && s < (uint32_t)A.n;
  const float4* __restrict__ rec = reinterpret_cast<const float4*>(A.rec);
  const float4* __restrict__ lo = A.rec_lo;
  uint32_t m = 0, cnt = 0, off = 0;
  float csx = 0.f, csy = 0.f, csz = 0.f;
  if (valid) {
    off = A.nl_off[s];
    m = A.smeta[s];  // sorted copy: no gather through the particle's tag
    const SysDev& S = A.sys[meta_sys(m)];
    Q.ri[lane] = rec[s];
    Q.li[lane] = lo[s];
    csx = S.cs_f[0]; csy = S.cs_f[1]; csz = S.cs_f[2];
    cnt = A.nl_cnt[s];
  }
  Q.csx[lane] = csx; Q.csy[lane] = csy; Q.csz[lane] = csz;
  // prefix sums of the list lengths over the warp
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const uint32_t pre = incl - cnt;
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  // the warp's entries are one contiguous run of the packed lists (from its first slot's start)
  const uint32_t* __restrict__ list =
      A.nl_pk + (int64_t)(s0 & ~31u) * (uint32_t)A.nl_max + __shfl_sync(0xffffffffu, off, 0);
  float fx = 0.f, fy = 0.f, fz = 0.f, u = 0.f;
  // evaluate the k queued pairs from queue position q0 (k <= 32); each particle adds its run in order
  auto drain = [&](uint32_t q0, uint32_t k) {
    __syncwarp();
    const bool have = (uint32_t)lane < k;
    uint32_t ow = 0;
    if (have) {
      const uint32_t x = Q.q[q0 + lane];
      ow = Q.own[x];
      const uint32_t code = Q.code[x];
      const float4 ro = Q.ri[ow], lio = Q.li[ow];
      const float4 rj = Q.sr[x], lj = Q.sl[x];
      const int dz = (int)(code / 9u) - 1, dy = (int)(code / 3u % 3u) - 1, dx = (int)(code % 3u) - 1;
      const uint32_t qt = (RecT<float>::bits(ro) & 7u) * kMaxTypes + (RecT<float>::bits(rj) & 7u);
      AccTerm t;
      const bool in = acc_pair(tab, qt, ro, lio, rj, lj, (float)dx * Q.csx[ow], (float)dy * Q.csy[ow],
                               (float)dz * Q.csz[ow], t);
      Q.sr[x] = make_float4(t.fr, t.dx.h, t.dy.h, t.dz.h);
      Q.sl[x] = make_float4(t.dx.l, t.dy.l, t.dz.l, t.v);
      Q.in[x] = in ? 1 : 0;
    }
    // runs: a queue position starts one where its particle differs from the previous position's
    const uint32_t prev = __shfl_up_sync(0xffffffffu, ow, 1);
    const bool start = have && (lane == 0 || prev != ow);
    const uint32_t starts = __ballot_sync(0xffffffffu, start);
    Q.runn[lane] = 0;
    __syncwarp();
    if (start) {
      const uint32_t after = starts & ~((2u << lane) - 1u);  // starts above this one
      const uint32_t next = after ? (uint32_t)(__ffs(after) - 1) : k;
      Q.run0[ow] = (uint8_t)lane;
      Q.runn[ow] = (uint8_t)(next - lane);
    }
    __syncwarp();
    const uint32_t r0 = Q.run0[lane], rn = Q.runn[lane];
    const uint32_t longest = __reduce_max_sync(0xffffffffu, rn);
    for (uint32_t j = 0; j < longest; ++j) {
      if (j < rn) {
        const uint32_t x = Q.q[q0 + r0 + j];
        if (Q.in[x]) {
          const float4 a = Q.sr[x], b = Q.sl[x];
          acc_add(a.x, DF{a.y, b.x}, DF{a.z, b.y}, DF{a.w, b.z}, b.w, fx, fy, fz, u);
        }
      }
    }
    __syncwarp();
  };
  for (uint32_t c = 0; c < total; c += (uint32_t)kNlqStage) {
    // the particle of each position p (the highest lane whose prefix is <= p) and its list entry
    uint32_t e[kNlqGroup];
#pragma unroll
    for (int g = 0; g < kNlqGroup; ++g) {
      const uint32_t p = c + 32u * g + (uint32_t)lane;
      uint32_t ow = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t cand = ow + (uint32_t)step;
        const uint32_t pc = __shfl_sync(0xffffffffu, pre, (int)(cand & 31u));
        if (cand < 32u && pc <= p) ow = cand;
      }
      Q.own[32 * g + lane] = (uint8_t)ow;
      e[g] = p < total ? list[p] : 0u;
    }
    // the entries' records and low parts to shared memory, all in flight together
    __syncwarp();  // the previous group's evaluations have read their staged pairs
#pragma unroll
    for (int g = 0; g < kNlqGroup; ++g) {
      const uint32_t p = c + 32u * g + (uint32_t)lane;
      if (p < total) {
        const uint32_t x = 32u * g + (uint32_t)lane;
        Q.code[x] = (uint8_t)(e[g] & 31u);
        cp_async16(&Q.sr[x], &rec[e[g] >> 5]);
        cp_async16(&Q.sl[x], &lo[e[g] >> 5]);
      }
    }
    cp_async_wait_all();
    // screen on the high parts; queue the pairs that pass, in order
    uint32_t qn = 0;
#pragma unroll
    for (int g = 0; g < kNlqGroup; ++g) {
      const uint32_t p = c + 32u * g + (uint32_t)lane;
      const uint32_t x = 32u * g + (uint32_t)lane;
      bool hit = false;
      if (p < total) {
        const uint32_t ow = Q.own[x], code = Q.code[x];
        const float4 ro = Q.ri[ow], rj = Q.sr[x];
        const int dz = (int)(code / 9u) - 1, dy = (int)(code / 3u % 3u) - 1, dx = (int)(code % 3u) - 1;
        const float ddx = ro.x - rj.x - (float)dx * Q.csx[ow], ddy = ro.y - rj.y - (float)dy * Q.csy[ow],
                    ddz = ro.z - rj.z - (float)dz * Q.csz[ow];
        const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        hit = r2 < tab.acc.rc2m[(RecT<float>::bits(ro) & 7u) * kMaxTypes + (RecT<float>::bits(rj) & 7u)];
      }
      const uint32_t mask = __ballot_sync(0xffffffffu, hit);
      if (hit) Q.q[qn + __popc(mask & ((1u << lane) - 1u))] = (uint8_t)x;
      qn += __popc(mask);
    }
    for (uint32_t q0 = 0; q0 < qn; q0 += 32u) drain(q0, min(32u, qn - q0));
  }
  if (!valid) return;
  const uint32_t tag = A.stag[s];
  if (BONDS || WALLS) bonded_terms<float>(A, A.sys[meta_sys(m)], tag, m, BONDS, WALLS, fx, fy, fz, u);
  store_f<float>(A.f, tag, fx, fy, fz, u);
}

// Bend-angle forces (and energy shares) added to the pair kernel's output.
template <typename R>
__global__ void k_bend(DevArrays A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const SysDev& S = A.sys[meta_sys(A.meta[i])];
  if (!has_bends(S)) return;
  R f[3], v;
  bend_on<R>(A, S, i, f, v);
  using V = typename V4<R>::T;
  V* fv = reinterpret_cast<V*>(A.f);
  V q = fv[i];
  q.x += f[0]; q.y += f[1]; q.z += f[2]; q.w += v;
  fv[i] = q;
}

// L lanes of one warp share one particle: lane q walks the stencil cells
// q, q+L, q+2L, ... of the 27, so each lane's chain of dependent loads is L
// times shorter; the lanes' partial sums are combined by a fixed xor-shuffle
// tree (the summation order, hence every bit of the result, is fixed).
template <typename R, bool BONDS, bool WALLS, bool EXCL, int L>
__global__ void __launch_bounds__(256) k_pair_lanes(DevArrays A) {
  __shared__ PairTab<R> tab;
  load_tab<R>(tab, A.types);
  __syncthreads();
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t s = (uint32_t)(g / L);
  const int q = (int)(g % L);
  const bool valid = s < (uint32_t)A.n;
  using Rec = typename RecT<R>::T;
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(A.rec);
  const uint32_t* __restrict__ scell = A.scell;
  const uint32_t* __restrict__ start = A.start;
  R fx = 0, fy = 0, fz = 0, u = 0;
  uint32_t tag = 0, m = 0;
  const SysDev* Sp = A.sys;
  if (valid) {
    tag = A.stag[s];
    const uint32_t cell = scell[s];
    const Rec ri = rec[s];
    const float4 li = rec_lo_at<R>(A.rec_lo, s);
    const uint32_t bi = RecT<R>::bits(ri);
    const uint32_t ti = bi & 7u, moli = bi >> 3;
    m = A.meta[tag];
    const uint32_t sid = meta_sys(m);
    Sp = &A.sys[sid];
    const SysDev& S = *Sp;
    int c[3];
    cell_decode(S, cell, c[0], c[1], c[2]);
    const R csx = sizeof(R) == 4 ? (R)S.cs_f[0] : (R)S.cs[0];
    const R csy = sizeof(R) == 4 ? (R)S.cs_f[1] : (R)S.cs[1];
    const R csz = sizeof(R) == 4 ? (R)S.cs_f[2] : (R)S.cs[2];
    bool prune = S.slab > 0.f && meta_con(m) && A.sys_free[sid] == 0;
    float nhx = 0.f, nhy = 0.f, nhz = 0.f, reach = 0.f, on = 0.f;
    if (prune) {
      const float ox = (float)ri.x, oy = (float)ri.y, oz = (float)ri.z;
      const float rx = S.grid_lo_f[0] + ((float)c[0] + 0.5f) * S.cs_f[0] + ox - S.c_f[0];
      const float ry = S.grid_lo_f[1] + ((float)c[1] + 0.5f) * S.cs_f[1] + oy - S.c_f[1];
      const float rz = S.grid_lo_f[2] + ((float)c[2] + 0.5f) * S.cs_f[2] + oz - S.c_f[2];
      surf_grad_f(S, rx, ry, rz, nhx, nhy, nhz);
      const float nn = fmaf(nhx, nhx, fmaf(nhy, nhy, nhz * nhz));
      if (nn > 0.f) {
        const float inv = rsqrtf(nn);
        nhx *= inv; nhy *= inv; nhz *= inv;
        reach = 0.5f * (S.cs_f[0] * fabsf(nhx) + S.cs_f[1] * fabsf(nhy) + S.cs_f[2] * fabsf(nhz)) + S.slab;
        on = nhx * ox + nhy * oy + nhz * oz;
      } else {
        prune = false;
      }
    }
    for (int k = q; k < 27; k += L) {
      const int dz = k / 9 - 1, dy = (k / 3) % 3 - 1, dx = k % 3 - 1;
      int x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
      if (x < 0 || x >= S.nc[0]) {
        if (!S.periodic[0]) continue;
        x = (x + S.nc[0]) % S.nc[0];
      }
      if (y < 0 || y >= S.nc[1]) {
        if (!S.periodic[1]) continue;
        y = (y + S.nc[1]) % S.nc[1];
      }
      if (z < 0 || z >= S.nc[2]) {
        if (!S.periodic[2]) continue;
        z = (z + S.nc[2]) % S.nc[2];
      }
      if (prune) {
        const float dist = nhx * (float)dx * S.cs_f[0] + nhy * (float)dy * S.cs_f[1] +
                           nhz * (float)dz * S.cs_f[2] - on;
        if (fabsf(dist) > reach) continue;
      }
      const uint32_t nb = cell_id(S, x, y, z);
      const uint32_t b = bucket_of(nb, A.hashed, A.log_t);
      const uint32_t t1 = start[b + 1];
      const R shx = (R)dx * csx, shy = (R)dy * csy, shz = (R)dz * csz;
      for (uint32_t t = start[b]; t < t1; ++t) {
        const Rec rj = rec[t];
        const uint32_t cj = A.rec_cell ? RecT<R>::bits(rj) >> 3 : scell[t];
        if (cj != nb || t == s) continue;
        const uint32_t bj = RecT<R>::bits(rj);
        if (EXCL && (bj >> 3) == moli) continue;
        const uint32_t qt = ti * kMaxTypes + (bj & 7u);
        pair_term<R>(tab, qt, ri, li, rj, A.rec_lo, t, shx, shy, shz, fx, fy, fz, u);
      }
    }
  }
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
    u += __shfl_xor_sync(0xffffffffu, u, o);
  }
  if (!valid || q != 0) return;
  if (BONDS || WALLS) bonded_terms<R>(A, *Sp, tag, m, BONDS, WALLS, fx, fy, fz, u);
  store_f<R>(A.f, tag, fx, fy, fz, u);
}

// ---------------------------------------------------------------------------
// Cell-tiled pair kernel (bucket = cell id, no hashing). Warp w evaluates
// the particles of its run of A.pair_tile (8, 16 or 32) sorted slots, one
// cell at a time: the run splits at cell boundaries into pieces of p particles
// of one home cell. For each piece the warp stages the records of the home
// cell's 27-cell stencil in shared memory, each shifted into the frame of the
// home cell, and the piece's particles share the lanes: p groups of
// L = floor(32/p) lanes, lane j of a group walking the staged candidates j,
// j + L, ...; a fixed segmented shuffle tree adds each group's partial
// sums. A candidate's record is read from global memory once per
// piece instead of once per particle, the stencil's bucket bounds once per
// piece, and the lanes walk one shared list in step; every warp has the same
// number of particles whatever the cells' occupancy. The pieces leave their
// pair forces in shared memory; then every lane adds the bonded terms of its
// own slot and stores the force, so the float64 bond arithmetic runs on all
// the run's lanes at once (the float64 pipe costs the same per warp
// instruction whatever the number of active lanes).
// Each lane tests a segment of 32 of its candidates against the home
// particle's largest cutoff first, one bit per hit in a register mask, then
// evaluates the pair terms over the set bits (self and same-molecule pairs
// are dropped there): the lanes of a warp run the Lennard-Jones arithmetic
// together instead of once per candidate that any lane finds in range.
// ---------------------------------------------------------------------------
constexpr int kTileWarps = 4;   // warps per CTA
constexpr int kTileSlots = 32;  // most sorted slots (particles) per warp: one per lane
// staged candidates per warp and window (256 float4 or 128 double4 records,
// 4 KB a warp)
template <typename R> constexpr int tile_cap() { return sizeof(R) == 4 ? 256 : 128; }

// Copy the staged candidates [w0, w0 + len) of one cell into the warp's
// stage. Lane k < 27 holds stencil cell k's first slot t0 and its staged
// offset pre (exclusive prefix of the counts). Four loads per lane are in
// flight before their stores. All 32 lanes call this.
template <typename R>
__device__ __forceinline__ void tile_stage(const typename RecT<R>::T* __restrict__ rec, typename RecT<R>::T* stage,
                                           uint32_t* code, uint32_t t0, uint32_t pre, R csx, R csy, R csz,
                                           uint32_t w0, uint32_t len, int lane) {
  using Rec = typename RecT<R>::T;
  constexpr int U = 4;
  for (uint32_t e0 = 0; e0 < len; e0 += 32u * U) {
    Rec r[U];
    int kk[U];
    uint32_t ts[U];
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const uint32_t e = e0 + 32u * v + (uint32_t)lane, g = w0 + e;
      // stencil cell of candidate g: the last k < 27 with pre_k <= g
      int k = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t pk = __shfl_sync(0xffffffffu, pre, k + step);
        if (k + step < 27 && pk <= g) k += step;
      }
      kk[v] = k;
      const uint32_t tk = __shfl_sync(0xffffffffu, t0, k), pk = __shfl_sync(0xffffffffu, pre, k);
      ts[v] = tk + (g - pk);
      if (e < len) r[v] = rec[ts[v]];
    }
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const uint32_t e = e0 + 32u * v + (uint32_t)lane;
      if (e < len) {
        const int k = kk[v];
        Rec q = r[v];
        q.x += (R)(k % 3 - 1) * csx;
        q.y += (R)((k / 3) % 3 - 1) * csy;
        q.z += (R)(k / 9 - 1) * csz;
        stage[e] = q;
        code[e] = ts[v] << 5 | (uint32_t)k;  // the candidate's slot and stencil cell
      }
    }
  }
}

// One piece: the particles in sorted slots [lo, hi) of home cell `home`;
// their pair forces (and energy shares) go to fw[0 .. hi - lo).
template <typename R, bool EXCL>
__device__ __forceinline__ void tile_piece(const DevArrays& A, const PairTab<R>& tab,
                                           const typename RecT<R>::T* __restrict__ rec, typename RecT<R>::T* stage,
                                           uint32_t* code, typename V4<R>::T* fw, uint32_t home, uint32_t lo,
                                           uint32_t hi, int lane) {
  using Rec = typename RecT<R>::T;
  const uint32_t* __restrict__ start = A.start;
  const SysDev& S = A.nsys == 1 ? A.sys[0] : A.sys[meta_sys(A.meta[A.stag[lo]])];
  int cx, cy, cz;
  cell_decode(S, home, cx, cy, cz);
  // lane k < 27: stencil cell (dx, dy, dz) = (k % 3, k / 3 % 3, k / 9) - 1
  uint32_t t0 = 0, cnt = 0;
  if (lane < 27) {
    int x = cx + lane % 3 - 1, y = cy + (lane / 3) % 3 - 1, z = cz + lane / 9 - 1;
    bool ok = true;
    if (x < 0 || x >= S.nc[0]) {
      ok = ok && S.periodic[0];
      x = (x + S.nc[0]) % S.nc[0];
    }
    if (y < 0 || y >= S.nc[1]) {
      ok = ok && S.periodic[1];
      y = (y + S.nc[1]) % S.nc[1];
    }
    if (z < 0 || z >= S.nc[2]) {
      ok = ok && S.periodic[2];
      z = (z + S.nc[2]) % S.nc[2];
    }
    if (ok) {
      const uint32_t nb = cell_id(S, x, y, z);
      t0 = start[nb];
      cnt = start[nb + 1] - t0;
    }
  }
  const R csx = sizeof(R) == 4 ? (R)S.cs_f[0] : (R)S.cs[0];
  const R csy = sizeof(R) == 4 ? (R)S.cs_f[1] : (R)S.cs[1];
  const R csz = sizeof(R) == 4 ? (R)S.cs_f[2] : (R)S.cs[2];
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const uint32_t pre = incl - cnt;
  const uint32_t M = __shfl_sync(0xffffffffu, incl, 31);
  // the home cell is stencil cell 13 (periodic axes have at least 3 cells,
  // so no other stencil cell is the home cell); its first slot is t0 there
  const uint32_t self0 = __shfl_sync(0xffffffffu, pre, 13) + lo - __shfl_sync(0xffffffffu, t0, 13);
  const uint32_t p = hi - lo;  // 1..kTileSlots
  const uint32_t L = 32u / p;  // lanes per particle: p L of the 32 lanes work
  const uint32_t g = (uint32_t)lane / L, lj = (uint32_t)lane - g * L;
  const bool act = g < p;
  const uint32_t s = lo + (act ? g : 0u);
  const Rec ri = rec[s];
  const float4 li = rec_lo_at<R>(A.rec_lo, s);
  const uint32_t bi = RecT<R>::bits(ri);
  const uint32_t ti = bi & 7u, moli = bi >> 3;
  const uint32_t self = self0 + g;
  R rcm = 0;  // largest squared cutoff of the particle's type (the mixed path's screen bound)
#pragma unroll
  for (int b = 0; b < kMaxTypes; ++b)
    rcm = max(rcm, sizeof(R) == 4 ? (R)tab.acc.rc2m[ti * kMaxTypes + b] : tab.rc2[ti * kMaxTypes + b]);
  R fx = 0, fy = 0, fz = 0, u = 0;
  for (uint32_t w0 = 0; w0 < M; w0 += (uint32_t)tile_cap<R>()) {
    const uint32_t len = min(M - w0, (uint32_t)tile_cap<R>());
    __syncwarp();
    tile_stage<R>(rec, stage, code, t0, pre, csx, csy, csz, w0, len, lane);
    __syncwarp();
    if (act) {
      // the lane's candidates are e = lj + i L, i < ne
      const uint32_t ne = len > lj ? (len - lj + L - 1u) / L : 0u;
      for (uint32_t i0 = 0; i0 < ne; i0 += 32u) {
        const uint32_t nseg = min(ne - i0, 32u);
        uint32_t mask = 0;
#pragma unroll 4
        for (uint32_t i = 0; i < nseg; ++i) {
          const Rec rj = stage[lj + (i0 + i) * L];
          const R ddx = ri.x - rj.x, ddy = ri.y - rj.y, ddz = ri.z - rj.z;
          const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
          if (r2 < rcm) mask |= 1u << i;
        }
        while (mask) {
          const uint32_t e = lj + (i0 + (uint32_t)(__ffs(mask) - 1)) * L;
          mask &= mask - 1u;
          if (w0 + e == self) continue;
          const Rec rj = stage[e];
          const uint32_t bj = RecT<R>::bits(rj);
          if (EXCL && (bj >> 3) == moli) continue;
          const uint32_t qt = ti * kMaxTypes + (bj & 7u);
          const R ddx = ri.x - rj.x, ddy = ri.y - rj.y, ddz = ri.z - rj.z;
          const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
          if constexpr (sizeof(R) == 4) {
            // the screen passed on the staged (shifted) record: the candidate's own record, low
            // part and stencil shift give the pair term
            if (r2 < tab.acc.rc2m[qt]) {
              const uint32_t cd = code[e], t = cd >> 5;
              const int k = (int)(cd & 31u);
              lj_term_acc(tab, qt, ri, li, rec[t], A.rec_lo[t], (float)(k % 3 - 1) * csx,
                          (float)((k / 3) % 3 - 1) * csy, (float)(k / 9 - 1) * csz, fx, fy, fz, u);
            }
          } else {
            if (r2 < tab.rc2[qt]) lj_term<R>(tab, qt, r2, ddx, ddy, ddz, fx, fy, fz, u);
          }
        }
      }
    }
  }
  // segmented tree: after offset o, lane j of a group holds the sum of its
  // group's lanes j .. min(j + 2o, L) - 1; lane 0 ends with the group's sum
  for (uint32_t o = 1; o < L; o <<= 1) {
    const R ox = __shfl_down_sync(0xffffffffu, fx, o), oy = __shfl_down_sync(0xffffffffu, fy, o);
    const R oz = __shfl_down_sync(0xffffffffu, fz, o), ou = __shfl_down_sync(0xffffffffu, u, o);
    if (lj + o < L) {
      fx += ox;
      fy += oy;
      fz += oz;
      u += ou;
    }
  }
  if (act && lj == 0) {
    typename V4<R>::T q;
    q.x = fx;
    q.y = fy;
    q.z = fz;
    q.w = u;
    fw[g] = q;
  }
  __syncwarp();  // the stage is rewritten for the next piece
}

template <typename R, bool BONDS, bool WALLS, bool EXCL>
__global__ void __launch_bounds__(kTileWarps * 32, sizeof(R) == 4 ? 6 : 4) k_pair_cell(DevArrays A) {
  using Rec = typename RecT<R>::T;
  __shared__ PairTab<R> tab;
  __shared__ Rec stage_all[kTileWarps][tile_cap<R>()];
  __shared__ uint32_t code_all[kTileWarps][tile_cap<R>()];
  __shared__ typename V4<R>::T f_all[kTileWarps][kTileSlots];
  load_tab<R>(tab, A.types);
  __syncthreads();
  const int lane = (int)(threadIdx.x & 31u);
  const uint32_t wib = threadIdx.x >> 5;
  const Rec* __restrict__ rec = reinterpret_cast<const Rec*>(A.rec);
  const uint64_t n = (uint64_t)A.n;
  const uint32_t slots = (uint32_t)A.pair_tile;  // 8, 16 or 32 particles per warp
  const uint64_t r0 = ((uint64_t)blockIdx.x * kTileWarps + wib) * slots;
  if (r0 >= n) return;  // warp-uniform
  const uint32_t r1 = (uint32_t)min(r0 + (uint64_t)slots, n);
  const uint64_t s = r0 + (uint64_t)lane;
  const bool mine = (uint32_t)lane < slots && s < n;
  uint32_t c = 0;
  bool first = false;
  if (mine) {
    c = A.scell[s];
    first = lane == 0 || A.scell[s - 1] != c;
  }
  uint32_t cut = __ballot_sync(0xffffffffu, first);  // piece starts: bit 0 is always set
  while (cut) {
    const int a = __ffs(cut) - 1;
    cut &= cut - 1u;
    const uint32_t lo = (uint32_t)r0 + (uint32_t)a;
    const uint32_t hi = cut ? (uint32_t)r0 + (uint32_t)(__ffs(cut) - 1) : r1;
    const uint32_t home = __shfl_sync(0xffffffffu, c, a);
    tile_piece<R, EXCL>(A, tab, rec, stage_all[wib], code_all[wib], f_all[wib] + (lo - (uint32_t)r0), home, lo,
                        hi, lane);
  }
  if (mine) {  // the pieces' leaders wrote f_all before the last __syncwarp
    const typename V4<R>::T q = f_all[wib][lane];
    R fx = q.x, fy = q.y, fz = q.z, u = q.w;
    const uint32_t tag = A.stag[s];
    if (BONDS || WALLS) {
      const uint32_t m = A.meta[tag];
      bonded_terms<R>(A, A.sys[meta_sys(m)], tag, m, BONDS, WALLS, fx, fy, fz, u);
    }
    store_f<R>(A.f, tag, fx, fy, fz, u);
  }
}

// No pair term anywhere: only bonds and walls, in particle order.
template <typename R>
__global__ void k_nopair(DevArrays A, int bonds, int walls) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const uint32_t m = A.meta[i];
  const SysDev& S = A.sys[meta_sys(m)];
  R fx = 0, fy = 0, fz = 0, u = 0;
  if (bonds || walls) bonded_terms<R>(A, S, (uint32_t)i, m, bonds, walls, fx, fy, fz, u);
  store_f<R>(A.f, (uint32_t)i, fx, fy, fz, u);
}

// ---------------------------------------------------------------------------
// integrator
// ---------------------------------------------------------------------------
// g at a point, keeping what the gradient needs (the gradient is formed only
// when a Newton update needs it).
struct GEval {
  double g, ux, uy, uz, q;
};

__device__ __forceinline__ GEval surf_g(const SysDev& S, double x, double y, double z) {
  GEval e;
  double dx = x - S.c[0], dy = y - S.c[1], dz = z - S.c[2];
  e.q = 0.0;
  switch (S.kind) {
    case kPlane:
      e.g = fma(S.p[0], dx, fma(S.p[1], dy, S.p[2] * dz));
      break;
    case kSphere:
      e.g = fma(dx, dx, fma(dy, dy, fma(dz, dz, -S.p[0] * S.p[0])));
      break;
    case kEllipsoid:
      dx *= S.inv_a2[0];  // keep a_d^-2 (x_d - c_d)
      dy *= S.inv_a2[1];
      dz *= S.inv_a2[2];
      e.g = fma(dx, x - S.c[0], fma(dy, y - S.c[1], fma(dz, z - S.c[2], -1.0)));
      break;
    case kTorus: {
      const double rho2 = fma(dx, dx, dy * dy);
      const double ir = nr_rsqrt(rho2);
      const double t = fma(rho2, ir, -S.p[0]);  // rho - R
      e.q = 2.0 * t * ir;
      e.g = fma(t, t, fma(dz, dz, -S.p[1] * S.p[1]));
      break;
    }
    case kBump: {
      if (S.periodic[0]) dx = wrap_min_image(dx, S.box_len[0]);
      if (S.periodic[1]) dy = wrap_min_image(dy, S.box_len[1]);
      const double w2 = S.p[1] * S.p[1];
      const double ex = S.p[0] * exp(-fma(dx, dx, dy * dy) / (2.0 * w2));
      e.q = ex / w2;
      e.g = dz - ex;
      break;
    }
    case kCylinder:
      if (S.axis == 0) dx = 0.0;
      else if (S.axis == 1) dy = 0.0;
      else dz = 0.0;
      e.g = fma(dx, dx, fma(dy, dy, fma(dz, dz, -S.p[0] * S.p[0])));
      break;
    default:
      e.g = 0.0;
  }
  e.ux = dx; e.uy = dy; e.uz = dz;
  return e;
}

// g at (x, y, z) on a held thylakoid piece; the gradient is kept in (ux, uy, uz).
__device__ __forceinline__ GEval thyl_geval(const SysDev& S, const Piece& q, double x, double y, double z) {
  GEval e;
  e.q = 0.0;
  e.g = thyl_eval(S, q, x, y, z, e.ux, e.uy, e.uz);
  return e;
}

__device__ __forceinline__ void surf_n(const SysDev& S, const GEval& e, double& nx, double& ny, double& nz) {
  switch (S.kind) {
    case kThylakoid: nx = e.ux; ny = e.uy; nz = e.uz; break;
    case kPlane: nx = S.p[0]; ny = S.p[1]; nz = S.p[2]; break;
    case kTorus: nx = e.q * e.ux; ny = e.q * e.uy; nz = 2.0 * e.uz; break;
    case kBump: nx = e.q * e.ux; ny = e.q * e.uy; nz = 1.0; break;
    case kSphere:
    case kEllipsoid:
    case kCylinder: nx = 2.0 * e.ux; ny = 2.0 * e.uy; nz = 2.0 * e.uz; break;
    default: nx = ny = nz = 0.0;
  }
}

// Float32 gradient from the pieces surf_g kept (offsets in float64).
__device__ __forceinline__ void surf_n_f(const SysDev& S, const GEval& e, float& nx, float& ny, float& nz) {
  switch (S.kind) {
    case kThylakoid: nx = d2f_rn(e.ux); ny = d2f_rn(e.uy); nz = d2f_rn(e.uz); break;
    case kPlane: nx = S.p_f[0]; ny = S.p_f[1]; nz = S.p_f[2]; break;
    case kTorus: {
      const float q = d2f_rn(e.q);
      nx = q * d2f_rn(e.ux); ny = q * d2f_rn(e.uy); nz = 2.f * d2f_rn(e.uz);
      break;
    }
    case kBump: {
      const float q = d2f_rn(e.q);
      nx = q * d2f_rn(e.ux); ny = q * d2f_rn(e.uy); nz = 1.f;
      break;
    }
    case kSphere:
    case kEllipsoid:
    case kCylinder: nx = 2.f * d2f_rn(e.ux); ny = 2.f * d2f_rn(e.uy); nz = 2.f * d2f_rn(e.uz); break;
    default: nx = ny = nz = 0.f;
  }
}

template <typename R> struct Force3 { R x, y, z; };

template <typename R> __device__ __forceinline__ Force3<R> load_f3(const void* f, int64_t i);
template <> __device__ __forceinline__ Force3<float> load_f3<float>(const void* f, int64_t i) {
  const float4 v = reinterpret_cast<const float4*>(f)[i];
  return {v.x, v.y, v.z};
}
template <> __device__ __forceinline__ Force3<double> load_f3<double>(const void* f, int64_t i) {
  const double4_32a v = reinterpret_cast<const double4_32a*>(f)[i];
  return {v.x, v.y, v.z};
}

template <typename R> __device__ __forceinline__ R sys_gamma(const SysDev& S);
template <> __device__ __forceinline__ float sys_gamma<float>(const SysDev& S) { return S.gamma_f; }
template <> __device__ __forceinline__ double sys_gamma<double>(const SysDev& S) { return S.gamma; }
template <typename R> __device__ __forceinline__ R sys_comb(const SysDev& S);
template <> __device__ __forceinline__ float sys_comb<float>(const SysDev& S) { return S.comb_f; }
template <> __device__ __forceinline__ double sys_comb<double>(const SysDev& S) { return S.comb; }
template <typename R> __device__ __forceinline__ R noise_amp(const SysDev& S, const TypeTable* T, uint32_t ty);
template <> __device__ __forceinline__ float noise_amp<float>(const SysDev& S, const TypeTable* T, uint32_t ty) {
  return S.noise_unit_f * T->sqrt_mass_f[ty];
}
template <> __device__ __forceinline__ double noise_amp<double>(const SysDev& S, const TypeTable* T, uint32_t ty) {
  return S.noise_unit * T->sqrt_mass[ty];
}

// Algorithm S1 force combination at step k for one particle, in R:
//   first step after a set state:  F = f - gamma p + f_r^k
//   otherwise:  F = [f - gamma p^{k-1/2} + (f_r^k + f_r^{k-1})/2] / (1 + gamma dt/2)
// with f_r = sqrt(2 m kT gamma / dt) xi, xi drawn from Philox in R. Float32
// only: with a slot xi, the normals of step k are stored there, and those of
// step k-1 read from it when xi_prev (they were stored by the previous step:
// the same values gauss3 would give again).
template <typename R>
__device__ __forceinline__ Force3<R> combine(const SysDev& S, const TypeTable* T, uint32_t ty, uint32_t pid,
                                             unsigned long long k, int mode, Force3<R> f, R px, R py, R pz,
                                             float4* xi = nullptr, bool xi_prev = false) {
  R nx = 0, ny = 0, nz = 0;
  const R amp = noise_amp<R>(S, T, ty);
  if (amp > (R)0) {
    R gx, gy, gz;
    gauss3(S.seed_lo, S.replica, pid, k, gx, gy, gz);
    if (mode == 0) {
      nx = amp * gx; ny = amp * gy; nz = amp * gz;
    } else {
      R hx, hy, hz;
      if constexpr (sizeof(R) == 4) {
        if (xi_prev) {
          const float4 w = *xi;
          hx = w.x; hy = w.y; hz = w.z;
        } else {
          gauss3(S.seed_lo, S.replica, pid, k - 1ull, hx, hy, hz);
        }
      } else {
        gauss3(S.seed_lo, S.replica, pid, k - 1ull, hx, hy, hz);
      }
      const R ha = (R)0.5 * amp;
      nx = ha * (gx + hx); ny = ha * (gy + hy); nz = ha * (gz + hz);
    }
    if constexpr (sizeof(R) == 4) {
      if (xi) *xi = make_float4(gx, gy, gz, 0.f);
    }
  }
  const R gam = sys_gamma<R>(S);
  Force3<R> F;
  F.x = f.x - gam * px + nx;
  F.y = f.y - gam * py + ny;
  F.z = f.z - gam * pz + nz;
  if (mode != 0) {
    const R c = sys_comb<R>(S);
    F.x *= c; F.y *= c; F.z *= c;
  }
  return F;
}

// Momentum half of Algorithm 1 at x^k: p^k = p^{k-1/2} + h (F - mu n) with
// n.p^k = 0. The residual is linear in (p, mu), so the Newton iteration ends
// after one exact step: the projection p - (n.p / n.n) n.
__device__ __forceinline__ void momentum_half(double h, double Fx, double Fy, double Fz, bool con, double nx,
                                              double ny, double nz, double inv_nn, double& px, double& py,
                                              double& pz) {
  px = fma(h, Fx, px); py = fma(h, Fy, py); pz = fma(h, Fz, pz);
  if (con) {
    const double sc = fma(nx, px, fma(ny, py, nz * pz)) * inv_nn;
    px = fma(-sc, nx, px); py = fma(-sc, ny, py); pz = fma(-sc, nz, pz);
  }
}

__device__ __forceinline__ bool finite_bits(double v) {
  return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000;
}

// Where the integrator puts the cell of x^{k+1}: nowhere (no pair forces),
// the handle's global bucket counters, or (resident engine) one system's
// counters in shared memory. put() records the cell and the particle's rank
// in its bucket (the order of the atomic; the bucket build makes it canonical).
struct NoBin {
  static constexpr bool kOn = false, kPos = false;
  __device__ __forceinline__ explicit NoBin(const DevArrays&) {}
  __device__ __forceinline__ void put(int64_t, uint32_t) const {}
  __device__ __forceinline__ void pos(int64_t, double, double, double) const {}
};
struct GlobalBin {
  static constexpr bool kOn = true, kPos = false;
  __device__ __forceinline__ void pos(int64_t, double, double, double) const {}
  uint32_t* cell;
  uint32_t* rank;
  uint32_t* count;
  int hashed, log_t;
  __device__ __forceinline__ explicit GlobalBin(const DevArrays& A)
      : cell(A.cell), rank(A.rank), count(A.count), hashed(A.hashed), log_t(A.log_t) {}
  __device__ __forceinline__ void put(int64_t i, uint32_t c) const {
    cell[i] = c;
    rank[i] = atomicAdd(&count[bucket_of(c, hashed, log_t)], 1u);
  }
};

// Neighbour-list mode: the particle keeps its cell until the next rebuild;
// its record moves with it (record at the build + the float64 displacement
// since the build; on the mixed path the sum is formed as a double-float and
// split again into the high and low parts), and a displacement beyond skin / 2
// raises the rebuild flag for this step's cell-list kernels.
template <typename R> struct NlSink {
  static constexpr bool kOn = false, kPos = true;
  using Rec = typename RecT<R>::T;
  const uint32_t* slot_of;
  const double* xb;
  const Rec* rec0;
  const float4* rec0_lo;
  Rec* rec;
  float4* rec_lo;
  uint32_t* dirty;
  float half_skin2;
  int64_t n;
  __device__ __forceinline__ explicit NlSink(const DevArrays& A)
      : slot_of(A.slot_of), xb(A.xb), rec0(reinterpret_cast<const Rec*>(A.rec0)), rec0_lo(A.rec0_lo),
        rec(reinterpret_cast<Rec*>(A.rec)), rec_lo(A.rec_lo), dirty(A.nl_dirty), half_skin2(A.nl_half_skin2),
        n(A.n) {}
  __device__ __forceinline__ void put(int64_t, uint32_t) const {}
  __device__ __forceinline__ void pos(int64_t i, double xn, double yn, double zn) const {
    const uint32_t s = slot_of[i];
    const double dx = xn - xb[i], dy = yn - xb[n + i], dz = zn - xb[2 * n + i];
    Rec r = rec0[i];
    float d2;
    if constexpr (sizeof(R) == 4) {
      const float4 l = rec0_lo[i];
      const DF ex = df_from(dx), ey = df_from(dy), ez = df_from(dz);
      const DF ox = df_add(DF{r.x, l.x}, ex), oy = df_add(DF{r.y, l.y}, ey), oz = df_add(DF{r.z, l.z}, ez);
      r.x = ox.h; r.y = oy.h; r.z = oz.h;
      rec_lo[s] = make_float4(ox.l, oy.l, oz.l, 0.f);
      d2 = fmaf(ex.h, ex.h, fmaf(ey.h, ey.h, ez.h * ez.h));
    } else {
      r.x += dx; r.y += dy; r.z += dz;
      d2 = d2f_rn(fma(dx, dx, fma(dy, dy, dz * dz)));
    }
    rec[s] = r;
    if (!(d2 <= half_skin2)) atomicOr(dirty, 1u);
  }
};

// Float64 path: combine + momentum half of step k + position half of step
// k+1, then the cell of x^{k+1} and its rank in the bucket counter.
//
// Position half of Algorithm 1: with y = x + (dt/m)(p + h F) and
// a = dt^2/(2m), x^{k+1} = y - a lambda n0 with n0 = grad g(x^k). After its
// first update the residual r_x of Algorithm 1 is zero, and the 4x4 Newton
// step reduces to lambda += g(x) / (a n1.n0), n1 = grad g(x) at the iterate
// (n1 = n0 for the frozen-normal variant). Stop when |g| < eta |n|, with
// |n| = |n0| (the two differ by |x - x^k| times the curvature), or when the
// update falls under 4 ulp of the position (round-off floor).
template <class Bin>
__device__ __forceinline__ void integrate_particle_fp64(const DevArrays& A, int64_t i, Force3<double> fr_in,
                                                        unsigned long long k, int mode, const Bin& bin) {
  const int64_t n = A.n;
  const uint32_t m = A.meta[i];
  const SysDev& S = A.sys[meta_sys(m)];
  const TypeTable* T = A.types;
  const uint32_t ty = meta_type(m);
  const double x = A.x[i], y = A.x[n + i], z = A.x[2 * n + i];
  double px = A.ph[i], py = A.ph[n + i], pz = A.ph[2 * n + i];
  const Force3<double> Fr = combine<double>(S, T, ty, (uint32_t)(i - S.first), k, mode, fr_in, px, py, pz);
  const double Fx = Fr.x, Fy = Fr.y, Fz = S.kind == kXY2D ? 0.0 : Fr.z;  // 2D plane: no z update
  const double h = S.half_dt;
  const bool con = meta_con(m);
  double n0x = 0.0, n0y = 0.0, n0z = 0.0, nn = 1.0, inv_nn = 0.0;
  Piece q0{};
  const bool held = S.kind == kThylakoid;  // composite surface: the piece at x^k for the whole solve
  if (con) {
    if (held) q0 = thyl_select(S, x, y, z);
    surf_n(S, held ? thyl_geval(S, q0, x, y, z) : surf_g(S, x, y, z), n0x, n0y, n0z);
    nn = fma(n0x, n0x, fma(n0y, n0y, n0z * n0z));
    inv_nn = nr_rcp(nn);
  }
  if (mode != 0) momentum_half(h, Fx, Fy, Fz, con, n0x, n0y, n0z, inv_nn, px, py, pz);
  double qx = fma(h, Fx, px), qy = fma(h, Fy, py), qz = fma(h, Fz, pz);  // p^{k+1/2} before the constraint
  const double dtm = S.dt * T->inv_mass[ty];
  double xn = fma(dtm, qx, x), yn = fma(dtm, qy, y), zn = fma(dtm, qz, z);
  if (con) {
    const double a = h * dtm;  // dt^2 / (2m)
    const double yx = xn, yy = yn, yz = zn;
    // |n1| and |n0| differ by about |x - x^k| times the curvature; the 2%
    // margin on g^2 keeps |g| / |n(x^{k+1})| below eta.
    const double tol2nn = 0.98 * S.tol2 * nn;
    const double inv_a_nn = S.frozen ? inv_nn * nr_rcp(a) : 0.0;
    double lam = 0.0;
    bool ok = false;
    for (int it = 0; it <= S.max_newton; ++it) {
      const GEval e = held ? thyl_geval(S, q0, xn, yn, zn) : surf_g(S, xn, yn, zn);
      if (e.g * e.g < tol2nn) {
        ok = true;
        break;
      }
      if (it == S.max_newton) break;
      double dl;
      if (S.frozen) {
        dl = e.g * inv_a_nn;
      } else {
        double n1x, n1y, n1z;
        surf_n(S, e, n1x, n1y, n1z);
        dl = e.g * nr_rcp(a * fma(n1x, n0x, fma(n1y, n0y, n1z * n0z)));
      }
      lam += dl;
      const double al = a * lam;
      xn = fma(-al, n0x, yx); yn = fma(-al, n0y, yy); zn = fma(-al, n0z, yz);
      if (it > 0) {  // round-off floor: the update is below 4 ulp of the position
        const double step = fabs(dl) * a * fmax(fabs(n0x), fmax(fabs(n0y), fabs(n0z)));
        if (step <= 4.0 * DBL_EPSILON * fmax(fabs(xn), fmax(fabs(yn), fabs(zn)))) {
          ok = true;
          break;
        }
      }
    }
    if (!ok) flag(A.status, kFlagRattle);
    const double hl = h * lam;
    qx = fma(-hl, n0x, qx); qy = fma(-hl, n0y, qy); qz = fma(-hl, n0z, qz);
  }
  if (!(finite_bits(xn) && finite_bits(yn) && finite_bits(zn) && finite_bits(qx) && finite_bits(qy) &&
        finite_bits(qz)))
    flag(A.status, kFlagNonfinite);
  A.x[i] = xn; A.x[n + i] = yn; A.x[2 * n + i] = zn;
  A.ph[i] = qx; A.ph[n + i] = qy; A.ph[2 * n + i] = qz;
  if constexpr (Bin::kPos) bin.pos(i, xn, yn, zn);
  if (Bin::kOn) {
    bool out = false;
    const uint32_t cell = cell_of_d(S, xn, yn, zn, out);
    if (out) flag(A.status, kFlagOutOfGrid);
    bin.put(i, cell);
  }
}

// ---------------------------------------------------------------------------
// Mixed path: float32 forces, noise and force combination; the position
// half, the momentum update and the surface normal of constrained particles
// in double-float arithmetic (df.cuh, about 48 significant bits, on the
// float32 pipe) from the float64 masters, which are read and written as
// float64.
//
// Algorithm 1 in multiplier form. The momentum half at x^k and the kick of the
// position half give q = p^{k-1/2} + dt F^k - s n0, s = n0.(p^{k-1/2} + h F^k)
// / |n0|^2, n0 = grad g(x^k); the position half then subtracts h lambda n0.
// Both corrections lie along n0, so with q0 = p^{k-1/2} + dt F^k,
// y = x^k + (dt/m) q0 and mu = (dt/m)(s + h lambda):
//   x^{k+1} = y - mu n0,   p^{k+1/2} = q0 - (m/dt) mu n0,   g(y - mu n0) = 0.
// The projection s only sets where the Newton iteration starts (mu_0 =
// (dt/m) s, formed in float32), not its root. On the first step after a state
// is set there is no momentum half: q0 = p^k + h F^k, mu_0 = 0.
//
// The position-half Newton update lambda += g / (a n1.n0) of Algorithm 1 reads
// mu += g(x(mu)) / (n1.n0) on the line x(mu) = y - mu n0 (mu = a lambda,
// n1 = grad g(x(mu)); n1 = n0 in the frozen-normal variant). g along the line
// is evaluated in double-float: for the quadrics (plane, sphere, ellipsoid,
// cylinder) by its exact line form g(y) - b mu + c mu^2 (b = grad g(y).n0,
// c = n0.H n0 / 2, H the constant Hessian), for the torus at the point
// itself; the Newton denominator n1.n0 is float32 (it scales the step, not
// the root). The other surfaces (Gaussian bump, thylakoid) take the float64
// form below. The full-step momentum p^k is not needed by the step and is
// formed only on read-out, with the float64 normal.
// ---------------------------------------------------------------------------

// Any surface by re-evaluation of g at x(mu) in float64 (Gaussian bump,
// thylakoid composite).
struct LineGeneric {
  const SysDev* S;
  double yx, yy, yz, n0x, n0y, n0z;
  float n0xf, n0yf, n0zf;
  Piece q;  // the held piece of a composite surface
  GEval e;
  __device__ __forceinline__ double g(double mu) {
    const double px = fma(-mu, n0x, yx), py = fma(-mu, n0y, yy), pz = fma(-mu, n0z, yz);
    e = S->kind == kThylakoid ? thyl_geval(*S, q, px, py, pz) : surf_g(*S, px, py, pz);
    return e.g;
  }
  __device__ __forceinline__ float n1n0(float) const {
    float n1x, n1y, n1z;
    surf_n_f(*S, e, n1x, n1y, n1z);
    return fmaf(n1x, n0xf, fmaf(n1y, n0yf, n1z * n0zf));
  }
};

// Newton on the line from mu_0: stop when |g| < tol_n (tolerance times |n0|,
// with a 1% margin for |n(x^{k+1})| != |n0|) or when an update falls under the
// round-off floor (4 ulp of the position).
template <class L>
__device__ __forceinline__ bool newton_line(L& line, int max_newton, bool frozen, float nnf, float tol_n,
                                            float floor_mu, float mu0f, double& mu) {
  mu = f2d(mu0f);
  double g = line.g(mu);
  for (int it = 0; it <= max_newton; ++it) {
    const float gf = d2f_rn(g);
    if (fabsf(gf) < tol_n) return true;
    if (it == max_newton) break;
    const float rden = __frcp_rn(frozen ? nnf : line.n1n0(d2f_rn(mu)));
    mu = fma(g, f2d(rden), mu);
    if (it > 0 && fabsf(gf * rden) <= floor_mu) return true;
    g = line.g(mu);
  }
  return false;
}

__device__ __forceinline__ bool df_surface(int32_t kind) {
  return kind == kPlane || kind == kSphere || kind == kEllipsoid || kind == kCylinder || kind == kTorus;
}

// g on the line x(mu) = y - mu n0 in double-float, D = y - c, N = n0.
// Quadrics: the line form g(y) - b mu + c mu^2. Torus: g at the point, with
// rho - R, rho and x(mu) - c kept in float32 for the Newton denominator.
struct DFTorusEval {
  float ttf, rhof, e0, e1, e2;
  __device__ __forceinline__ DF g(const SysDev& S, const DF D[3], const DF N[3], DF mu) {
    DF E[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) E[d] = df_sub(D[d], df_mul(N[d], mu));
    const DF rho = df_sqrt(df_add(df_mul(E[0], E[0]), df_mul(E[1], E[1])));
    const DF t = df_sub(rho, S.R_df);
    ttf = t.h;
    rhof = rho.h;
    e0 = E[0].h; e1 = E[1].h; e2 = E[2].h;
    return df_add(df_add(df_mul(t, t), df_mul(E[2], E[2])), S.gconst_df);
  }
  // n1.n0 = 2 (rho - R)/rho (e_xy . n0_xy) + 2 e_z n0_z
  __device__ __forceinline__ float n1n0(const DF N[3]) const {
    return 2.f * ttf / rhof * fmaf(e0, N[0].h, e1 * N[1].h) + 2.f * e2 * N[2].h;
  }
};

// Position half of a constrained particle on a plane, sphere, ellipsoid,
// cylinder or torus (multiplier form above): reads x^k, p^{k-1/2} (or p^k on
// the first step) and the combined force F, returns x^{k+1} and p^{k+1/2}.
// y - c, n0 = grad g(x^k) and g in double-float. For the quadrics the Newton
// iteration runs on the line form first in float32, which brings mu to
// float32 resolution (about 1e-7 of mu n0, itself about 1e-4 sigma), then
// continues in double-float until g, evaluated in double-float, meets the
// tolerance; the torus iterates in double-float throughout. x^{k+1} =
// c + (y - c) - mu n0 is rounded once to float64; p^{k+1/2} = p + (kick F -
// (m/dt) mu n0) adds a float32 increment to the float64 momentum.
__device__ __forceinline__ void position_half_df(const SysDev& S, uint32_t ty, int mode, const double xv[3],
                                                 const double pv[3], const float pf[3], const float F[3],
                                                 uint32_t* status, double xo[3], double qo[3]) {
  DF D[3], N[3];
  const DF kick = mode ? S.dt_df : S.half_dt_df;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const DF q0 = df_add(df_from(pv[d]), df_mul_f(kick, F[d]));  // q0 = p + kick F
    const DF X = df_from(xv[d]);
    N[d] = S.c_zero ? X : df_sub(X, S.c_df[d]);                   // x - c (n0 below)
    D[d] = df_add(N[d], df_mul(S.dtm_df[ty], q0));               // y - c = x - c + (dt/m) q0
  }
  DF gy{0.f, 0.f}, b{0.f, 0.f};
  float c = 0.f;
  switch (S.kind) {
    case kPlane:
#pragma unroll
      for (int d = 0; d < 3; ++d) N[d] = S.pn_df[d];
      gy = df_dot3(S.pn_df, D);
      b = df_dot3(S.pn_df, N);
      break;
    case kEllipsoid: {
      DF U[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        N[d] = df_scale2(df_mul(N[d], S.inv_a2_df[d]), 2.f);
        U[d] = df_mul(D[d], S.inv_a2_df[d]);
        c = fmaf(N[d].h * N[d].h, S.inv_a2_df[d].h, c);
      }
      gy = df_add_f(df_dot3(U, D), -1.f);
      b = df_scale2(df_dot3(U, N), 2.f);
      break;
    }
    case kTorus: {
      const DF rho = df_sqrt(df_add(df_mul(N[0], N[0]), df_mul(N[1], N[1])));
      const DF q = df_scale2(df_div(df_sub(rho, S.R_df), rho), 2.f);  // 2 (rho - R) / rho
      N[0] = df_mul(q, N[0]);
      N[1] = df_mul(q, N[1]);
      N[2] = df_scale2(N[2], 2.f);
      break;
    }
    default: {  // sphere; cylinder without the axis component (n0 has none)
      DF M[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const bool off = S.kind == kCylinder && d == S.axis;
        M[d] = off ? DF{0.f, 0.f} : D[d];
        N[d] = off ? DF{0.f, 0.f} : df_scale2(N[d], 2.f);
      }
      gy = df_add(df_dot3(M, M), S.gconst_df);
      b = df_scale2(df_dot3(M, N), 2.f);
      break;
    }
  }
  const float nnf = fmaf(N[0].h, N[0].h, fmaf(N[1].h, N[1].h, N[2].h * N[2].h));
  if (S.kind == kSphere || S.kind == kCylinder) c = nnf;
  float mu0 = 0.f;
  if (mode) {  // mu_0 = (dt/m) n0.(p + h F) / |n0|^2
    float sp = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) sp = fmaf(N[d].h, fmaf(S.half_dt_f, F[d], pf[d]), sp);
    mu0 = S.dtm_f[ty] * sp / nnf;
  }
  const float tol_n = 0.99f * S.tol_f * sqrtf(nnf);
  // round-off floor: an update below 4 units of the double-float resolution of the position
  const float dmax = fmaxf(fabsf(D[0].h), fmaxf(fabsf(D[1].h), fabsf(D[2].h)));
  const float floor_mu = 4.f * 0x1p-47f * dmax / fmaxf(fabsf(N[0].h), fmaxf(fabsf(N[1].h), fabsf(N[2].h)));
  const bool torus = S.kind == kTorus;
  int it = 0;
  if (!torus) {  // float32 Newton on the line form g(y) - b mu + c mu^2
    for (; it < S.max_newton; ++it) {
      const float gf = fmaf(fmaf(c, mu0, -b.h), mu0, gy.h);
      if (fabsf(gf) < 0.5f * tol_n) break;
      const float dmu = gf * __frcp_rn(S.frozen ? nnf : fmaf(-2.f * mu0, c, b.h));
      mu0 += dmu;
      if (fabsf(dmu) <= 0x1p-22f * fabsf(mu0)) {
        ++it;
        break;
      }
    }
  }
  DFTorusEval T;
  DF mu = {mu0, 0.f};
  DF g = torus ? T.g(S, D, N, mu) : df_add_f(df_sub(gy, df_mul(b, mu)), c * mu.h * mu.h);
  bool ok = false;
  for (;; ++it) {
    if (fabsf(g.h) < tol_n) { ok = true; break; }
    if (it >= S.max_newton) break;
    const float den = S.frozen ? nnf : (torus ? T.n1n0(N) : fmaf(-2.f * mu.h, c, b.h));
    const float dmu = g.h * __frcp_rn(den);
    mu = df_add_f(mu, dmu);
    if (it > 0 && fabsf(dmu) <= floor_mu) { ok = true; break; }
    g = torus ? T.g(S, D, N, mu) : df_add_f(df_sub(gy, df_mul(b, mu)), c * mu.h * mu.h);
  }
  if (!ok) flag(status, kFlagRattle);
  const float kickf = mode ? S.dt_df.h : S.half_dt_df.h;
  const float cm = mu.h * S.inv_dtm_df[ty].h;  // (m/dt) mu
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    DF e = df_sub(D[d], df_mul(N[d], mu));  // (y - c) - mu n0
    if (!S.c_zero) e = df_add(e, S.c_df[d]);
    xo[d] = df_to(e);
    qo[d] = pv[d] + f2d(fmaf(kickf, F[d], -cm * N[d].h));  // p + kick F - (m/dt) mu n0
  }
}

template <class Bin>
__device__ __forceinline__ void integrate_particle_mixed(const DevArrays& A, int64_t i, Force3<float> fr_in,
                                                         unsigned long long k, int mode, const Bin& bin,
                                                         float4* xi = nullptr, bool xi_prev = false) {
  const int64_t n = A.n;
  const uint32_t m = A.meta[i];
  const SysDev& S = A.sys[meta_sys(m)];
  const uint32_t ty = meta_type(m);
  const double x = A.x[i], y = A.x[n + i], z = A.x[2 * n + i];
  const double px = A.ph[i], py = A.ph[n + i], pz = A.ph[2 * n + i];
  const float pxf = d2f_rn(px), pyf = d2f_rn(py), pzf = d2f_rn(pz);
  Force3<float> F =
      combine<float>(S, A.types, ty, (uint32_t)(i - S.first), k, mode, fr_in, pxf, pyf, pzf, xi, xi_prev);
  if (S.kind == kXY2D) F.z = 0.f;  // 2D plane: no z update
  double xn, yn, zn, qx, qy, qz;
  if (meta_con(m) && df_surface(S.kind)) {
    const double xv[3] = {x, y, z}, pv[3] = {px, py, pz};
    const float pf[3] = {pxf, pyf, pzf}, Fv[3] = {F.x, F.y, F.z};
    double xo[3], qo[3];
    position_half_df(S, ty, mode, xv, pv, pf, Fv, A.status, xo, qo);
    xn = xo[0]; yn = xo[1]; zn = xo[2];
    qx = qo[0]; qy = qo[1]; qz = qo[2];
  } else {
    const double kick = mode ? S.dt : S.half_dt;
    qx = fma(kick, f2d(F.x), px); qy = fma(kick, f2d(F.y), py); qz = fma(kick, f2d(F.z), pz);
    const double dtm = S.dtm[ty];
    const double yx = fma(dtm, qx, x), yy = fma(dtm, qy, y), yz = fma(dtm, qz, z);
    xn = yx; yn = yy; zn = yz;
    if (meta_con(m)) {  // Gaussian bump, thylakoid: float64 line
      const float xf = d2f_rn(x), yf = d2f_rn(y), zf = d2f_rn(z);
      float n0xf, n0yf, n0zf;
      Piece q0{};
      if (S.kind == kThylakoid) {  // composite surface: the piece at x^k, held for the solve
        q0 = thyl_select(S, x, y, z);
        double gx, gy, gz;
        thyl_eval(S, q0, x, y, z, gx, gy, gz);
        n0xf = d2f_rn(gx); n0yf = d2f_rn(gy); n0zf = d2f_rn(gz);
      } else {
        surf_grad_f(S, xf - S.c_f[0], yf - S.c_f[1], zf - S.c_f[2], n0xf, n0yf, n0zf);
      }
      const float nnf = fmaf(n0xf, n0xf, fmaf(n0yf, n0yf, n0zf * n0zf));
      float mu0f = 0.f;
      if (mode) {  // mu_0 = (dt/m) n0.(p + h F) / |n0|^2
        const float hf = S.half_dt_f;
        const float sp =
            fmaf(n0xf, fmaf(hf, F.x, pxf), fmaf(n0yf, fmaf(hf, F.y, pyf), n0zf * fmaf(hf, F.z, pzf)));
        mu0f = S.dtm_f[ty] * sp / nnf;
      }
      const float tol_n = 0.99f * S.tol_f * sqrtf(nnf);
      const float floor_mu = 4.f * (float)DBL_EPSILON * fmaxf(fabsf(xf), fmaxf(fabsf(yf), fabsf(zf))) /
                             fmaxf(fabsf(n0xf), fmaxf(fabsf(n0yf), fabsf(n0zf)));
      LineGeneric L;
      L.S = &S;
      L.yx = yx; L.yy = yy; L.yz = yz;
      L.n0x = f2d(n0xf); L.n0y = f2d(n0yf); L.n0z = f2d(n0zf);
      L.n0xf = n0xf; L.n0yf = n0yf; L.n0zf = n0zf;
      L.q = q0;
      double mu;
      if (!newton_line(L, S.max_newton, S.frozen, nnf, tol_n, floor_mu, mu0f, mu)) flag(A.status, kFlagRattle);
      xn = fma(-mu, L.n0x, yx); yn = fma(-mu, L.n0y, yy); zn = fma(-mu, L.n0z, yz);
      const double c = mu * S.inv_dtm[ty];
      qx = fma(-c, L.n0x, qx); qy = fma(-c, L.n0y, qy); qz = fma(-c, L.n0z, qz);
    }
  }
  if (!(finite_bits(xn) && finite_bits(yn) && finite_bits(zn) && finite_bits(qx) && finite_bits(qy) &&
        finite_bits(qz)))
    flag(A.status, kFlagNonfinite);
  A.x[i] = xn; A.x[n + i] = yn; A.x[2 * n + i] = zn;
  A.ph[i] = qx; A.ph[n + i] = qy; A.ph[2 * n + i] = qz;
  if constexpr (Bin::kPos) bin.pos(i, xn, yn, zn);
  if (Bin::kOn) {
    bool out = false;
    const uint32_t cell = cell_of_f(S, xn, yn, zn, out);
    if (out) flag(A.status, kFlagOutOfGrid);
    bin.put(i, cell);
  }
}

template <typename R>
__global__ void __launch_bounds__(256, 4) k_integrate_nl(DevArrays A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const unsigned long long k = *A.step;
  const int mode = *A.mode;
  const NlSink<R> bin(A);
  if constexpr (sizeof(R) == 4) {
    const bool store = A.noise && A.store_noise;
    float4* xi = store ? A.noise + i : nullptr;
    const bool xi_prev = store && k > 0ull && *A.noise_k == k - 1ull;  // ~0: none stored
    integrate_particle_mixed(A, i, load_f3<float>(A.f, i), k, mode, bin, xi, xi_prev);
  } else {
    integrate_particle_fp64(A, i, load_f3<double>(A.f, i), k, mode, bin);
  }
}

template <typename R, bool BIN>
__global__ void __launch_bounds__(256, 4) k_integrate(DevArrays A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const unsigned long long k = *A.step;
  const int mode = *A.mode;
  using Bin = typename std::conditional<BIN, GlobalBin, NoBin>::type;
  const Bin bin(A);
  if constexpr (sizeof(R) == 4) integrate_particle_mixed(A, i, load_f3<float>(A.f, i), k, mode, bin);
  else integrate_particle_fp64(A, i, load_f3<double>(A.f, i), k, mode, bin);
}

// ---------------------------------------------------------------------------
// Resident engine. One CTA takes one whole system from the work list and
// advances it J.nsteps time steps with the system's cell list (bucket starts,
// sorted ids, cells and records) and its forces in shared memory; positions
// and momenta stay in global memory, read and written once per step. The
// per-particle code is the global kernels' own (pair_slot, the integrators,
// cell_offsets), the stencil visits the cells in the same order and each cell
// lists its particles by id as in the global buckets, so every force sum and
// every update is the same: the two engines give the same bits. Buckets are
// per system (res_t of them, dense or hashed on local cell ids).
// ---------------------------------------------------------------------------
template <typename R> struct SharedCells {
  using Rec = typename RecT<R>::T;
  const Rec* rec_;
  const float4* lo_;
  const uint32_t* scell_;
  const uint32_t* start_;
  const uint16_t* stag_;
  uint32_t first, base;
  int hashed, log_t;
  __device__ __forceinline__ const float4* lo() const { return lo_; }
  __device__ __forceinline__ uint32_t tag(uint32_t s) const { return first + stag_[s]; }
  __device__ __forceinline__ uint32_t scell(uint32_t t) const { return scell_[t]; }
  __device__ __forceinline__ Rec rec(uint32_t t) const { return rec_[t]; }
  __device__ __forceinline__ uint32_t start(uint32_t b) const { return start_[b]; }
  __device__ __forceinline__ uint32_t bucket(uint32_t cell) const { return bucket_of(cell - base, hashed, log_t); }
};

// The cell of particle li is kept in word li * stride of the x-force array
// (stride = sizeof(R) / 4), the slot where the same thread has just read the
// particle's force: the two are never live at the same time.
struct SharedBin {
  static constexpr bool kOn = true, kPos = false;
  __device__ __forceinline__ void pos(int64_t, double, double, double) const {}
  uint32_t* cell;
  uint32_t stride;
  uint16_t* rank;
  uint32_t* count;
  int64_t first;
  uint32_t base;
  int hashed, log_t;
  __device__ __forceinline__ void put(int64_t i, uint32_t c) const {
    const uint32_t li = (uint32_t)(i - first);
    cell[li * stride] = c;
    rank[li] = (uint16_t)atomicAdd(&count[bucket_of(c - base, hashed, log_t)], 1u);
  }
};

// Bucket counters (s_start[0..T)) -> bucket starts, scatter, canonical order
// and records, for the n particles of the system starting at `first`.
template <typename R>
__device__ __forceinline__ void resident_cells(const DevArrays& A, const SysDev& S, int64_t first, uint32_t n,
                                               uint32_t T, uint32_t* s_start, const uint32_t* s_cell,
                                               uint32_t cstride, const uint16_t* s_rank, uint16_t* s_tmp,
                                               uint16_t* s_stag, uint32_t* s_scell, void* s_rec, float4* s_lo,
                                               uint32_t* warp_tot) {
  const uint32_t tid = threadIdx.x, bd = blockDim.x;
  {
    const uint32_t per = (T + bd - 1) / bd;
    const uint32_t lo = min(tid * per, T), hi = min(lo + per, T);
    uint32_t sum = 0;
    for (uint32_t e = lo; e < hi; ++e) sum += s_start[e];
    uint32_t total;
    uint32_t run = block_exclusive_scan(sum, warp_tot, total);
    for (uint32_t e = lo; e < hi; ++e) {
      const uint32_t c = s_start[e];
      s_start[e] = run;
      run += c;
    }
    if (tid == 0) s_start[T] = n;
  }
  __syncthreads();
  for (uint32_t li = tid; li < n; li += bd)
    s_tmp[s_start[bucket_of(s_cell[li * cstride] - S.cell_base, S.res_hashed, S.res_log_t)] + s_rank[li]] =
        (uint16_t)li;
  __syncthreads();
  const int64_t nn = A.n;
  for (uint32_t d = tid; d < n; d += bd) {
    const uint32_t li = s_tmp[d];
    const uint32_t c = s_cell[li * cstride];
    const uint32_t b = bucket_of(c - S.cell_base, S.res_hashed, S.res_log_t);
    const uint32_t s0 = s_start[b], s1 = s_start[b + 1];
    uint32_t r = 0;
    for (uint32_t t = s0; t < s1; ++t) r += (s_tmp[t] < li) ? 1u : 0u;
    const uint32_t dd = s0 + r;
    const int64_t i = first + li;
    const uint32_t m = A.meta[i];
    double o[3];
    cell_offsets(S, c, A.x[i], A.x[nn + i], A.x[2 * nn + i], o);
    const uint32_t mol = A.mol ? (uint32_t)A.mol[i] : 0u;
    s_stag[dd] = (uint16_t)li;
    s_scell[dd] = c;
    put_rec<R>(s_rec, s_lo, dd, o[0], o[1], o[2], meta_type(m) | ((A.rec_cell ? c : mol) << 3));
  }
  __syncthreads();
}

template <typename R, bool BONDS, bool WALLS, bool EXCL>
__global__ void __launch_bounds__(kResidentMaxThreads, 2) k_resident(DevArrays A, ResidentJob J) {
  using Rec = typename RecT<R>::T;
  __shared__ PairTab<R> tab;
  __shared__ uint32_t warp_tot[33];
  __shared__ int s_job;
  extern __shared__ __align__(32) unsigned char smem[];
  // Layout (nmax particles, tmax buckets): records (mixed path: then their
  // low parts), then the force components
  // (each nmax R; the x-forces double as the particles' cells and the
  // y-forces as the scatter's slot list, which are live only while the
  // forces are not), sorted cells, bucket counters / starts, sorted ids,
  // ranks. 32-byte alignment for the float64 path's double4 records (the
  // size carries 32 bytes of slack for this).
  const uint32_t mis = (uint32_t)__cvta_generic_to_shared(smem) & 31u;
  Rec* s_rec = reinterpret_cast<Rec*>(smem + (mis ? 32u - mis : 0u));
  float4* s_lo = reinterpret_cast<float4*>(s_rec + J.nmax);
  R* s_fx = reinterpret_cast<R*>(sizeof(R) == 4 ? reinterpret_cast<unsigned char*>(s_lo + J.nmax)
                                                : reinterpret_cast<unsigned char*>(s_rec + J.nmax));
  R* s_fy = s_fx + J.nmax;
  R* s_fz = s_fy + J.nmax;
  uint32_t* s_cell = reinterpret_cast<uint32_t*>(s_fx);
  constexpr uint32_t cstride = sizeof(R) / 4;
  uint16_t* s_tmp = reinterpret_cast<uint16_t*>(s_fy);
  uint32_t* s_scell = reinterpret_cast<uint32_t*>(s_fz + J.nmax);
  uint32_t* s_start = s_scell + J.nmax;  // bucket counters, then (after the scan) bucket starts
  uint16_t* s_stag = reinterpret_cast<uint16_t*>(s_start + J.tmax + 1);
  uint16_t* s_rank = s_stag + J.nmax;
  load_tab<R>(tab, A.types);
  const unsigned long long k0 = *A.step;
  const int mode0 = *A.mode;
  const uint32_t tid = threadIdx.x, bd = blockDim.x;
  const int64_t nn = A.n;
  for (;;) {
    __syncthreads();  // the previous system is finished by every thread
    if (tid == 0) s_job = (int)atomicAdd(J.next, 1u);
    __syncthreads();
    const int job = s_job;
    if (job >= J.nsys) break;
    const SysDev& S = A.sys[J.order[job]];
    const int64_t first = S.first;
    const uint32_t n = (uint32_t)S.n;
    const uint32_t T = S.res_t;
    const SharedBin bin{s_cell, cstride, s_rank, s_start, first, S.cell_base, S.res_hashed, S.res_log_t};
    const SharedCells<R> C{s_rec, s_lo, s_scell, s_start, s_stag, (uint32_t)first, S.cell_base, S.res_hashed,
                           S.res_log_t};
    // cell list of the positions the launch starts from
    for (uint32_t e = tid; e <= T; e += bd) s_start[e] = 0u;
    __syncthreads();
    for (uint32_t li = tid; li < n; li += bd) {
      const int64_t i = first + li;
      bool out = false;
      const uint32_t cell = cell_of<R>(S, A.x[i], A.x[nn + i], A.x[2 * nn + i], out);
      if (out) flag(A.status, kFlagOutOfGrid);
      bin.put(i, cell);
    }
    __syncthreads();
    resident_cells<R>(A, S, first, n, T, s_start, s_cell, cstride, s_rank, s_tmp, s_stag, s_scell, s_rec, s_lo,
                      warp_tot);
    for (int j = 0; j < J.nsteps; ++j) {
      for (uint32_t s = tid; s < n; s += bd) {
        R fx, fy, fz, u;
        const uint32_t li = pair_slot<R, BONDS, WALLS, EXCL>(A, C, tab, s, fx, fy, fz, u) - (uint32_t)first;
        s_fx[li] = fx;
        s_fy[li] = fy;
        s_fz[li] = fz;
      }
      __syncthreads();
      for (uint32_t e = tid; e <= T; e += bd) s_start[e] = 0u;  // the starts are not read again this step
      if (has_bends(S)) {
        for (uint32_t li = tid; li < n; li += bd) {
          R f[3], v;
          bend_on<R>(A, S, first + li, f, v);
          s_fx[li] += f[0];
          s_fy[li] += f[1];
          s_fz[li] += f[2];
        }
      }
      __syncthreads();
      const unsigned long long k = k0 + (unsigned long long)j;
      const int mode = j == 0 ? mode0 : 1;
      for (uint32_t li = tid; li < n; li += bd) {
        const Force3<R> f{s_fx[li], s_fy[li], s_fz[li]};
        if constexpr (sizeof(R) == 4) integrate_particle_mixed(A, first + li, f, k, mode, bin);
        else integrate_particle_fp64(A, first + li, f, k, mode, bin);
      }
      __syncthreads();
      // the last step's list would only be rebuilt by the next launch
      if (j + 1 < J.nsteps)
        resident_cells<R>(A, S, first, n, T, s_start, s_cell, cstride, s_rank, s_tmp, s_stag, s_scell, s_rec,
                          s_lo, warp_tot);
    }
  }
}

__global__ void k_advance_n(unsigned long long* step, int32_t* mode, int32_t nsteps) {
  *step += (unsigned long long)nsteps;
  *mode = 1;
}

size_t resident_smem_bytes(int precision, uint32_t nmax, uint32_t tmax) {
  const size_t rec = precision == 0 ? sizeof(double4_32a) : 2 * sizeof(float4);  // mixed: record + low part
  const size_t r = precision == 0 ? sizeof(double) : sizeof(float);
  return (size_t)nmax * (rec + 3 * r + sizeof(uint32_t) + 2 * sizeof(uint16_t)) +
         sizeof(uint32_t) * ((size_t)tmax + 1) + 32;
}

template <typename R, bool BONDS, bool WALLS, bool EXCL>
cudaError_t resident_one(const DevArrays& A, const ResidentJob& J, int threads, int grid_cap, cudaStream_t st) {
  const size_t smem = resident_smem_bytes(sizeof(R) == 4 ? 1 : 0, J.nmax, J.tmax);
  auto kern = k_resident<R, BONDS, WALLS, EXCL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = std::min(J.nsys, per_sm * sms);
  if (grid_cap > 0) grid = std::min(grid, grid_cap);
  kern<<<grid, threads, smem, st>>>(A, J);
  return cudaGetLastError();
}

cudaError_t launch_advance_n(const DevArrays& A, int32_t nsteps, cudaStream_t st) {
  k_advance_n<<<1, 1, 0, st>>>(A.step, A.mode, nsteps);
  return cudaGetLastError();
}

template <typename R>
cudaError_t resident_dispatch(const DevArrays& A, const ResidentJob& J, int bonds, int walls, int excl, int threads,
                              int grid_cap, cudaStream_t st) {
  const int key = (bonds ? 4 : 0) | (walls ? 2 : 0) | (excl ? 1 : 0);
  switch (key) {
    case 0: return resident_one<R, false, false, false>(A, J, threads, grid_cap, st);
    case 1: return resident_one<R, false, false, true>(A, J, threads, grid_cap, st);
    case 2: return resident_one<R, false, true, false>(A, J, threads, grid_cap, st);
    case 3: return resident_one<R, false, true, true>(A, J, threads, grid_cap, st);
    case 4: return resident_one<R, true, false, false>(A, J, threads, grid_cap, st);
    case 5: return resident_one<R, true, false, true>(A, J, threads, grid_cap, st);
    case 6: return resident_one<R, true, true, false>(A, J, threads, grid_cap, st);
    default: return resident_one<R, true, true, true>(A, J, threads, grid_cap, st);
  }
}

cudaError_t launch_resident(const DevArrays& A, int precision, const ResidentJob& J, int bonds, int walls, int excl,
                            int threads, int grid_cap, cudaStream_t st) {
  if (J.nsys <= 0 || J.nsteps <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(J.next, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  return precision == 0 ? resident_dispatch<double>(A, J, bonds, walls, excl, threads, grid_cap, st)
                        : resident_dispatch<float>(A, J, bonds, walls, excl, threads, grid_cap, st);
}

int resident_blocks_per_sm(int precision, int bonds, int walls, int excl, uint32_t nmax, uint32_t tmax, int threads) {
  const size_t smem = resident_smem_bytes(precision, nmax, tmax);
  int per_sm = 0;
  cudaError_t e;
  const int key = (bonds ? 4 : 0) | (walls ? 2 : 0) | (excl ? 1 : 0);
  auto q = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  };
  if (precision == 0) {
    switch (key) {
      case 0: e = q(k_resident<double, false, false, false>); break;
      case 1: e = q(k_resident<double, false, false, true>); break;
      case 2: e = q(k_resident<double, false, true, false>); break;
      case 3: e = q(k_resident<double, false, true, true>); break;
      case 4: e = q(k_resident<double, true, false, false>); break;
      case 5: e = q(k_resident<double, true, false, true>); break;
      case 6: e = q(k_resident<double, true, true, false>); break;
      default: e = q(k_resident<double, true, true, true>); break;
    }
  } else {
    switch (key) {
      case 0: e = q(k_resident<float, false, false, false>); break;
      case 1: e = q(k_resident<float, false, false, true>); break;
      case 2: e = q(k_resident<float, false, true, false>); break;
      case 3: e = q(k_resident<float, false, true, true>); break;
      case 4: e = q(k_resident<float, true, false, false>); break;
      case 5: e = q(k_resident<float, true, false, true>); break;
      case 6: e = q(k_resident<float, true, true, false>); break;
      default: e = q(k_resident<float, true, true, true>); break;
    }
  }
  return e == cudaSuccess ? per_sm : 0;
}

__global__ void k_advance(unsigned long long* step, int32_t* mode) {
  *step += 1ull;
  *mode = 1;
}

// p^k = momentum half of Algorithm 1 from p^{k-1/2} and F^k (state unchanged):
// the force combination as in k_integrate, the projection with the float64
// normal at x^k in both precisions.
template <typename R>
__global__ void k_finish(DevArrays A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (i >= n) return;
  const int mode = *A.mode;
  if (mode == 0) {
    A.pk[i] = A.ph[i]; A.pk[n + i] = A.ph[n + i]; A.pk[2 * n + i] = A.ph[2 * n + i];
    return;
  }
  const unsigned long long k = *A.step;
  const uint32_t m = A.meta[i];
  const SysDev& S = A.sys[meta_sys(m)];
  const uint32_t ty = meta_type(m);
  const double x = A.x[i], y = A.x[n + i], z = A.x[2 * n + i];
  double px = A.ph[i], py = A.ph[n + i], pz = A.ph[2 * n + i];
  Force3<R> Fr = combine<R>(S, A.types, ty, (uint32_t)(i - S.first), k, 1, load_f3<R>(A.f, i), (R)px, (R)py,
                            (R)pz);
  if (S.kind == kXY2D) Fr.z = (R)0;
  const bool con = meta_con(m);
  double nx = 0.0, ny = 0.0, nz = 0.0, inv_nn = 0.0;
  if (con) {  // the float64 normal in both precisions: n.p^k = 0 to float64 rounding
    surf_eval(S, x, y, z, nx, ny, nz);
    inv_nn = 1.0 / fma(nx, nx, fma(ny, ny, nz * nz));
  }
  momentum_half(S.half_dt, (double)Fr.x, (double)Fr.y, (double)Fr.z, con, nx, ny, nz, inv_nn, px, py, pz);
  A.pk[i] = px; A.pk[n + i] = py; A.pk[2 * n + i] = pz;
}

// ---------------------------------------------------------------------------
// read-out
// ---------------------------------------------------------------------------
__global__ void k_get_state(DevArrays A, double* xa, double* va, double* pa) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  if (i >= n) return;
  const double inv_m = A.types->inv_mass[meta_type(A.meta[i])];
  for (int d = 0; d < 3; ++d) {
    if (xa) xa[3 * i + d] = A.x[d * n + i];
    if (va) va[3 * i + d] = A.pk[d * n + i] * inv_m;
    if (pa) pa[3 * i + d] = A.ph[d * n + i];
  }
}

template <typename R>
__global__ void k_get_forces(DevArrays A, double* fa, double* ua) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  using V = typename V4<R>::T;
  const V v = reinterpret_cast<const V*>(A.f)[i];
  if (fa) {
    fa[3 * i] = (double)v.x;
    fa[3 * i + 1] = (double)v.y;
    fa[3 * i + 2] = (double)v.z;
  }
  if (ua) ua[i] = (double)v.w;
}


// Arithmetic peak probe: every thread runs 8 independent fused multiply-add
// chains of `iters` steps each in R; one result per thread is kept in a
// device sink so the chains cannot be dropped.
__device__ double g_peak_sink;

template <typename R>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, R b, R c) {
  R a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (R)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  R t = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += a[k];
  if (t == (R)-1.2345) g_peak_sink = (double)t;  // never true for these inputs; keeps the chains live
}

cudaError_t launch_fma_probe(int precision, int blocks, int iters, cudaStream_t st) {
  if (precision == 0) k_fma_probe<double><<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7);
  else k_fma_probe<float><<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-7f);
  return cudaGetLastError();
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Residuals of Section 2.2 (g = 0, n.v = 0): per-warp maxima, one atomic per warp.
__global__ void k_residual(DevArrays A, unsigned long long* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  double r0 = 0.0, r1 = 0.0, r2 = 0.0;
  if (i < n) {
    const uint32_t m = A.meta[i];
    if (meta_con(m)) {
      const SysDev& S = A.sys[meta_sys(m)];
      double nx, ny, nz;
      const double g = surf_eval(S, A.x[i], A.x[n + i], A.x[2 * n + i], nx, ny, nz);
      const double gn = sqrt(nx * nx + ny * ny + nz * nz);
      const double inv_m = A.types->inv_mass[meta_type(m)];
      const double nv = (nx * A.pk[i] + ny * A.pk[n + i] + nz * A.pk[2 * n + i]) * inv_m;
      r0 = fabs(g) / gn;
      r1 = fabs(g);
      r2 = fabs(nv) / gn;
    }
  }
  r0 = warp_max(r0);
  r1 = warp_max(r1);
  r2 = warp_max(r2);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&out[0], r0);
    atomic_max_nonneg(&out[1], r1);
    atomic_max_nonneg(&out[2], r2);
  }
}

// Per-system sums and maxima; a warp whose particles belong to one system
// reduces in registers and issues one atomic per quantity.
template <typename R>
__global__ void k_observables(DevArrays A, double* obs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  uint32_t sid = 0xffffffffu;
  if (i < n) {
    const uint32_t m = A.meta[i];
    sid = meta_sys(m);
    const SysDev& S = A.sys[sid];
    const double inv_m = A.types->inv_mass[meta_type(m)];
    const double px = A.pk[i], py = A.pk[n + i], pz = A.pk[2 * n + i];
    const double x = A.x[i], y = A.x[n + i], z = A.x[2 * n + i];
    const double dx = x - A.xref[i], dy = y - A.xref[n + i], dz = z - A.xref[2 * n + i];
    using V = typename V4<R>::T;
    const V f = reinterpret_cast<const V*>(A.f)[i];
    v[0] = 0.5 * (px * px + py * py + pz * pz) * inv_m;
    v[1] = (double)f.w;
    v[2] = dx * dx + dy * dy + dz * dz;
    if (S.kind == kSphere) {
      const double R2 = S.p[0] * S.p[0];
      v[3] = ((A.xref[i] - S.c[0]) * (x - S.c[0]) + (A.xref[n + i] - S.c[1]) * (y - S.c[1]) +
              (A.xref[2 * n + i] - S.c[2]) * (z - S.c[2])) / R2;
    }
    const bool con = meta_con(m);
    v[4] = (con || S.kind == kXY2D) ? 2.0 : 3.0;
    if (con) {
      double nx, ny, nz;
      const double g = surf_eval(S, x, y, z, nx, ny, nz);
      const double gn = sqrt(nx * nx + ny * ny + nz * nz);
      v[5] = fabs(g) / gn;
      v[6] = fabs((nx * px + ny * py + nz * pz) * inv_m) / gn;
    }
    v[7] = 1.0;
  }
  const uint32_t s0 = __shfl_sync(0xffffffffu, sid, 0);
  const bool uniform = __all_sync(0xffffffffu, sid == s0 || sid == 0xffffffffu);
  if (uniform) {
    if (s0 == 0xffffffffu) return;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (q == 5 || q == 6) ? warp_max(v[q]) : warp_sum(v[q]);
    if ((threadIdx.x & 31) != 0) return;
    sid = s0;
  } else if (sid == 0xffffffffu) {
    return;
  }
  double* o = obs + 8 * (int64_t)sid;
  for (int q = 0; q < 8; ++q) {
    if (q == 5 || q == 6) atomic_max_nonneg(reinterpret_cast<unsigned long long*>(&o[q]), v[q]);
    else if (v[q] != 0.0) atomicAdd(&o[q], v[q]);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// Threads per block of the per-particle step kernels: 256, or fewer (a
// multiple of 32) for small systems, so that the blocks spread over the SMs.
// An SM's float64 pipe retires two operations per clock, and a system of a
// thousand particles in 256-thread blocks would occupy four of them.
static int block_for(int64_t units) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v > 0 ? v : 1;
  }
  const int64_t per = (units + sms - 1) / sms;
  return (int)std::max<int64_t>(32, std::min<int64_t>(256, (per + 31) / 32 * 32));
}

cudaError_t launch_build_meta(const DevArrays& A, const int64_t* d_first, int nsys, const int32_t* d_type,
                              const uint8_t* d_con, const int32_t* d_mol, int, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  k_build_meta<<<grid_for(A.n, 256), 256, 0, st>>>(A, d_first, nsys, d_type, d_con, d_mol);
  return cudaGetLastError();
}

cudaError_t launch_set_state(const DevArrays& A, const double* d_x, const double* d_v, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  k_set_state<<<grid_for(A.n, 256), 256, 0, st>>>(A, d_x, d_v);
  return cudaGetLastError();
}

cudaError_t launch_restore(const DevArrays& A, const double* d_x, const double* d_ph, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  k_restore<<<grid_for(A.n, 256), 256, 0, st>>>(A, d_x, d_ph);
  return cudaGetLastError();
}

cudaError_t launch_bin(const DevArrays& A, int precision, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  const int b = block_for(A.n);
  if (precision == 0) k_bin<double><<<grid_for(A.n, b), b, 0, st>>>(A);
  else k_bin<float><<<grid_for(A.n, b), b, 0, st>>>(A);
  return cudaGetLastError();
}

static inline uint32_t scan_blocks_of(const DevArrays& A) {
  return (A.nbucket + kScanPerBlock - 1) / kScanPerBlock;
}

cudaError_t launch_scan(const DevArrays& A, int advance, cudaStream_t st) {
  k_scan_onepass<<<scan_blocks_of(A), kScanThreads, 0, st>>>(A, advance);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const DevArrays& A, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  k_scatter<<<grid_for(A.n, block_for(A.n)), block_for(A.n), 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_order(const DevArrays& A, const DevArrays& O, uint32_t coord_shift, uint32_t morton_drop,
                         uint32_t sys_shift, uint32_t* order, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  const OrderKey K{coord_shift, morton_drop, sys_shift};
  k_order_hist<<<grid_for(A.n, 256), 256, 0, st>>>(A, O, K);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_scan(O, 0, st);
  if (e != cudaSuccess) return e;
  k_order_scatter<<<grid_for(A.n, 256), 256, 0, st>>>(A, O, K, order);
  return cudaGetLastError();
}

cudaError_t launch_cells_after_bin(const DevArrays& A, int advance, cudaStream_t st) {
  cudaError_t e = launch_scan(A, advance, st);
  if (e == cudaSuccess) e = launch_scatter(A, st);
  return e;
}

cudaError_t launch_bucket_build(const DevArrays& A, int precision, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  const int b = block_for(A.n);
  if (precision == 0) k_bucket_build<double><<<grid_for(A.n, b), b, 0, st>>>(A);
  else k_bucket_build<float><<<grid_for(A.n, b), b, 0, st>>>(A);
  return cudaGetLastError();
}

template <typename R>
static void pair_dispatch_row(const DevArrays& A, int bonds, int walls, int excl, cudaStream_t st) {
  const int b = block_for(A.n);
  const unsigned g = grid_for(A.n, b);
  const int key = (bonds ? 4 : 0) | (walls ? 2 : 0) | (excl ? 1 : 0);
  switch (key) {
    case 0: k_pair_row<R, false, false, false><<<g, b, 0, st>>>(A); break;
    case 1: k_pair_row<R, false, false, true><<<g, b, 0, st>>>(A); break;
    case 2: k_pair_row<R, false, true, false><<<g, b, 0, st>>>(A); break;
    case 3: k_pair_row<R, false, true, true><<<g, b, 0, st>>>(A); break;
    case 4: k_pair_row<R, true, false, false><<<g, b, 0, st>>>(A); break;
    case 5: k_pair_row<R, true, false, true><<<g, b, 0, st>>>(A); break;
    case 6: k_pair_row<R, true, true, false><<<g, b, 0, st>>>(A); break;
    default: k_pair_row<R, true, true, true><<<g, b, 0, st>>>(A); break;
  }
}

template <typename R, int L>
static void pair_dispatch_l(const DevArrays& A, int bonds, int walls, int excl, cudaStream_t st) {
  const int b = block_for((int64_t)A.n * L);
  const unsigned g = grid_for((int64_t)A.n * L, b);
  const int key = (bonds ? 4 : 0) | (walls ? 2 : 0) | (excl ? 1 : 0);
  switch (key) {
    case 0: k_pair_lanes<R, false, false, false, L><<<g, b, 0, st>>>(A); break;
    case 1: k_pair_lanes<R, false, false, true, L><<<g, b, 0, st>>>(A); break;
    case 2: k_pair_lanes<R, false, true, false, L><<<g, b, 0, st>>>(A); break;
    case 3: k_pair_lanes<R, false, true, true, L><<<g, b, 0, st>>>(A); break;
    case 4: k_pair_lanes<R, true, false, false, L><<<g, b, 0, st>>>(A); break;
    case 5: k_pair_lanes<R, true, false, true, L><<<g, b, 0, st>>>(A); break;
    case 6: k_pair_lanes<R, true, true, false, L><<<g, b, 0, st>>>(A); break;
    default: k_pair_lanes<R, true, true, true, L><<<g, b, 0, st>>>(A); break;
  }
}

template <typename R>
static void pair_dispatch_cell(const DevArrays& A, int bonds, int walls, int excl, cudaStream_t st) {
  const uint64_t per_cta = (uint64_t)kTileWarps * (uint64_t)A.pair_tile;
  const unsigned g = (unsigned)std::max<uint64_t>(1, ((uint64_t)A.n + per_cta - 1) / per_cta);
  const int b = kTileWarps * 32;
  const int key = (bonds ? 4 : 0) | (walls ? 2 : 0) | (excl ? 1 : 0);
  switch (key) {
    case 0: k_pair_cell<R, false, false, false><<<g, b, 0, st>>>(A); break;
    case 1: k_pair_cell<R, false, false, true><<<g, b, 0, st>>>(A); break;
    case 2: k_pair_cell<R, false, true, false><<<g, b, 0, st>>>(A); break;
    case 3: k_pair_cell<R, false, true, true><<<g, b, 0, st>>>(A); break;
    case 4: k_pair_cell<R, true, false, false><<<g, b, 0, st>>>(A); break;
    case 5: k_pair_cell<R, true, false, true><<<g, b, 0, st>>>(A); break;
    case 6: k_pair_cell<R, true, true, false><<<g, b, 0, st>>>(A); break;
    default: k_pair_cell<R, true, true, true><<<g, b, 0, st>>>(A); break;
  }
}

template <typename R>
static void pair_dispatch(const DevArrays& A, int bonds, int walls, int excl, int lanes, cudaStream_t st) {
  if (A.pair_tile && !A.hashed) {
    pair_dispatch_cell<R>(A, bonds, walls, excl, st);
    return;
  }
  switch (lanes) {
    case 2: pair_dispatch_l<R, 2>(A, bonds, walls, excl, st); break;
    case 4: pair_dispatch_l<R, 4>(A, bonds, walls, excl, st); break;
    case 8: pair_dispatch_l<R, 8>(A, bonds, walls, excl, st); break;
    default: pair_dispatch_row<R>(A, bonds, walls, excl, st); break;
  }
}

template <typename R>
static void pair_dispatch_nl(const DevArrays& A, int bonds, int walls, cudaStream_t st) {
  const unsigned g = grid_for(A.n, 256);
  if constexpr (sizeof(R) == 4) {
    if (A.pair_queue) {
      const int64_t warps = (A.n + A.list_warp - 1) / A.list_warp;
      const unsigned gq = (unsigned)((warps + kQueueWarps - 1) / kQueueWarps);
      switch ((bonds ? 2 : 0) | (walls ? 1 : 0)) {
        case 0: k_pair_nlq<false, false><<<gq, kQueueWarps * 32, 0, st>>>(A); break;
        case 1: k_pair_nlq<false, true><<<gq, kQueueWarps * 32, 0, st>>>(A); break;
        case 2: k_pair_nlq<true, false><<<gq, kQueueWarps * 32, 0, st>>>(A); break;
        default: k_pair_nlq<true, true><<<gq, kQueueWarps * 32, 0, st>>>(A); break;
      }
      return;
    }
  }
  switch ((bonds ? 2 : 0) | (walls ? 1 : 0)) {
    case 0: k_pair_nl<R, false, false><<<g, 256, 0, st>>>(A); break;
    case 1: k_pair_nl<R, false, true><<<g, 256, 0, st>>>(A); break;
    case 2: k_pair_nl<R, true, false><<<g, 256, 0, st>>>(A); break;
    default: k_pair_nl<R, true, true><<<g, 256, 0, st>>>(A); break;
  }
}

cudaError_t launch_nl_build(const DevArrays& A, int precision, int excl, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  const unsigned g = grid_for(A.n, 256);
  if (precision == 0) {
    if (excl) k_nl_build<double, true><<<g, 256, 0, st>>>(A);
    else k_nl_build<double, false><<<g, 256, 0, st>>>(A);
  } else {
    if (excl) k_nl_build<float, true><<<g, 256, 0, st>>>(A);
    else k_nl_build<float, false><<<g, 256, 0, st>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_pair(const DevArrays& A, int precision, int has_pairs, int bonds, int walls, int excl,
                        cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  if (has_pairs && A.nl_dirty) {
    if (precision == 0) pair_dispatch_nl<double>(A, bonds, walls, st);
    else pair_dispatch_nl<float>(A, bonds, walls, st);
    return cudaGetLastError();
  }
  if (!has_pairs) {
    const int b = block_for(A.n);
    if (precision == 0) k_nopair<double><<<grid_for(A.n, b), b, 0, st>>>(A, bonds, walls);
    else k_nopair<float><<<grid_for(A.n, b), b, 0, st>>>(A, bonds, walls);
  } else if (precision == 0) {
    pair_dispatch<double>(A, bonds, walls, excl, A.pair_lanes, st);
  } else {
    pair_dispatch<float>(A, bonds, walls, excl, A.pair_lanes, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_bend(const DevArrays& A, int precision, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  const int b = block_for(A.n);
  if (precision == 0) k_bend<double><<<grid_for(A.n, b), b, 0, st>>>(A);
  else k_bend<float><<<grid_for(A.n, b), b, 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_integrate(const DevArrays& A, int precision, int has_pairs, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  const int b = block_for(A.n);
  const unsigned g = grid_for(A.n, b);
  if (A.nl_dirty && has_pairs) {
    if (precision == 0) k_integrate_nl<double><<<g, b, 0, st>>>(A);
    else k_integrate_nl<float><<<g, b, 0, st>>>(A);
  } else if (precision == 0) {
    if (has_pairs) k_integrate<double, true><<<g, b, 0, st>>>(A);
    else k_integrate<double, false><<<g, b, 0, st>>>(A);
  } else {
    if (has_pairs) k_integrate<float, true><<<g, b, 0, st>>>(A);
    else k_integrate<float, false><<<g, b, 0, st>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_advance(const DevArrays& A, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(A.step, A.mode);
  return cudaGetLastError();
}

cudaError_t launch_finish(const DevArrays& A, int precision, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  const int b = block_for(A.n);
  if (precision == 0) k_finish<double><<<grid_for(A.n, b), b, 0, st>>>(A);
  else k_finish<float><<<grid_for(A.n, b), b, 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_get_state(const DevArrays& A, double* xa, double* va, double* pa, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  k_get_state<<<grid_for(A.n, 256), 256, 0, st>>>(A, xa, va, pa);
  return cudaGetLastError();
}

__global__ void k_check_conversions(const double* __restrict__ in, int64_t n, float* __restrict__ out_f,
                                    double* __restrict__ out_d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float f = d2f_rn(in[i]);
  out_f[i] = f;
  out_d[i] = f2d(f);
}

cudaError_t launch_check_conversions(const double* in, int64_t n, float* out_f, double* out_d, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_check_conversions<<<grid_for(n, 256), 256, 0, st>>>(in, n, out_f, out_d);
  return cudaGetLastError();
}

cudaError_t launch_get_forces(const DevArrays& A, int precision, double* fa, double* ua, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  if (precision == 0) k_get_forces<double><<<grid_for(A.n, 256), 256, 0, st>>>(A, fa, ua);
  else k_get_forces<float><<<grid_for(A.n, 256), 256, 0, st>>>(A, fa, ua);
  return cudaGetLastError();
}

cudaError_t launch_residual(const DevArrays& A, unsigned long long* d_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_out, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess || A.n == 0) return e;
  k_residual<<<grid_for(A.n, 256), 256, 0, st>>>(A, d_out);
  return cudaGetLastError();
}

cudaError_t launch_observables(const DevArrays& A, int precision, double* d_obs, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_obs, 0, 8 * sizeof(double) * (size_t)A.nsys, st);
  if (e != cudaSuccess || A.n == 0) return e;
  if (precision == 0) k_observables<double><<<grid_for(A.n, 256), 256, 0, st>>>(A, d_obs);
  else k_observables<float><<<grid_for(A.n, 256), 256, 0, st>>>(A, d_obs);
  return cudaGetLastError();
}

}  // namespace surfmd
