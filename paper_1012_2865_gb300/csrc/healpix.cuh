// healpix.cuh -- nested-scheme pixel centres on the device (Step 3a of
// Sec. 3.1; HEALPix, Gorski et al. 2005).
//
// Geometry: 12 base faces (0-3 north, 4-7 equatorial, 8-11 south); in the
// projection plane (t = 4 phi / pi, u = 3 z / 2 in the equatorial belt) face
// centres sit at (2k+1, 1), (2k, 0) and (2k+1, -1); pixel (ix, iy) of a face
// sits at p1 = (ix+1/2)/Nside, p2 = (iy+1/2)/Nside along the two diagonals.
// The nested index interleaves ix (even bits) and iy (odd bits), so the
// children of p are 4p + {0,1,2,3} (Sec. 2.1).
//
// The azimuth is phi = (pi/2) * a / b with integers a, b; the quadrant is
// removed exactly, so components that vanish are exact zeros and
// mirror-symmetric pixels (phi = pi/4 + k pi/2) give |n_x| == |n_y| exactly.
// The FP64 version uses explicitly rounded operations (no FMA contraction),
// so its arithmetic is the same sequence of IEEE operations as a plain FP64
// evaluation of the same formulas.
#pragma once
#include <stdint.h>

namespace rtg {

__device__ __forceinline__ uint32_t compact_even_bits(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0f0f0f0fu;
  x = (x | (x >> 4)) & 0x00ff00ffu;
  x = (x | (x >> 8)) & 0x0000ffffu;
  return x;
}

// Integer description of a pixel's ring: polar (nr < nside, pole distance
// 1 - |z| = nr^2 / (3 nside^2)) or equatorial (z = zq / (3 nside)), azimuth
// numerator a and denominator b (phi = (pi/2) a / b, 0 <= a < 4b).
struct RingInt {
  int64_t nr;     // pixels per quadrant in the ring
  int64_t zq;     // equatorial: z = zq / (3 nside)
  int polar;      // 1 north cap, -1 south cap, 0 equatorial belt
  int64_t a, b;
};

__device__ __forceinline__ RingInt pixel_ring(int level, uint32_t pix) {
  const int64_t nside = (int64_t)1 << level;
  const uint32_t npface = (uint32_t)(nside * nside);
  const int face = (int)(pix / npface);
  const uint32_t ipf = pix - (uint32_t)face * npface;
  const int64_t ix = compact_even_bits(ipf);
  const int64_t iy = compact_even_bits(ipf >> 1);
  const int64_t s = ix + iy + 1;
  const int k = face & 3;
  RingInt R;
  int64_t tnum;
  if (face < 4) {
    if (s > nside) { R.polar = 1; R.nr = 2 * nside - s; R.zq = 0; }
    else { R.polar = 0; R.nr = nside; R.zq = 2 * s; }
    tnum = (2 * k + 1) * R.nr + ix - iy;
  } else if (face < 8) {
    R.polar = 0;
    R.nr = nside;
    R.zq = 2 * (s - nside);
    tnum = 2 * k * R.nr + ix - iy;
  } else {
    if (s < nside) { R.polar = -1; R.nr = s; R.zq = 0; }
    else { R.polar = 0; R.nr = nside; R.zq = 2 * (s - 2 * nside); }
    tnum = (2 * k + 1) * R.nr + ix - iy;
  }
  R.b = 2 * R.nr;
  int64_t a = tnum % (4 * R.b);
  if (a < 0) a += 4 * R.b;
  R.a = a;
  return R;
}

// FP64 unit vector; returns 1 if the pixel lies on a 45-degree meridian
// (|n_x| == |n_y| exactly).
__device__ __forceinline__ int pix2vec64(int level, uint32_t pix, double n[3]) {
  const RingInt R = pixel_ring(level, pix);
  const int64_t nside = (int64_t)1 << level;
  double z, st;
  if (R.polar != 0) {
    const double omz = __ddiv_rn((double)(R.nr * R.nr), (double)(3 * nside * nside));
    z = __dsub_rn(1.0, omz);
    if (R.polar < 0) z = -z;
    st = __dsqrt_rn(__dmul_rn(omz, __dsub_rn(2.0, omz)));
  } else {
    z = __ddiv_rn((double)R.zq, (double)(3 * nside));
    st = __dsqrt_rn(__dmul_rn(__dsub_rn(1.0, z), __dadd_rn(1.0, z)));
  }
  const int64_t q = R.a / R.b;
  const int64_t m = R.a - q * R.b;
  double c0, s0;
  int diag = 0;
  if (m == 0) {
    c0 = 1.0;
    s0 = 0.0;
  } else if (2 * m == R.b) {
    c0 = __dsqrt_rn(0.5);
    s0 = c0;
    diag = 1;
  } else if (2 * m < R.b) {
    const double ang = __dmul_rn(3.141592653589793 * 0.5, __ddiv_rn((double)m, (double)R.b));
    sincos(ang, &s0, &c0);
  } else {
    const double ang = __dmul_rn(3.141592653589793 * 0.5, __ddiv_rn((double)(R.b - m), (double)R.b));
    sincos(ang, &c0, &s0);
  }
  double c, s;
  switch (q) {
    case 0: c = c0; s = s0; break;
    case 1: c = -s0; s = c0; break;
    case 2: c = -c0; s = -s0; break;
    default: c = s0; s = -c0; break;
  }
  n[0] = __dmul_rn(st, c);
  n[1] = __dmul_rn(st, s);
  n[2] = z;
  return diag;
}

// FP32 unit vector for the mixed path.  Each component is within
// kDirErr32 of the FP64 vector above (absolute); zeros and 45-degree mirror
// symmetry are exact as in FP64.
constexpr float kDirErr32 = 16.0f * 5.9604645e-8f;  // 16 * 2^-24

__device__ __forceinline__ int pix2vec32(int level, uint32_t pix, float n[3]) {
  const RingInt R = pixel_ring(level, pix);
  const int64_t nside = (int64_t)1 << level;
  float z, st;
  if (R.polar != 0) {
    const float omz = (float)((double)(R.nr * R.nr) / (double)(3 * nside * nside));
    z = 1.0f - omz;
    if (R.polar < 0) z = -z;
    st = sqrtf(omz * (2.0f - omz));
  } else {
    z = (float)((double)R.zq / (double)(3 * nside));
    st = sqrtf((1.0f - z) * (1.0f + z));
  }
  const int64_t q = R.a / R.b;
  const int64_t m = R.a - q * R.b;
  float c0, s0;
  int diag = 0;
  if (m == 0) {
    c0 = 1.0f;
    s0 = 0.0f;
  } else if (2 * m == R.b) {
    c0 = 0.70710678118654752f;
    s0 = c0;
    diag = 1;
  } else if (2 * m < R.b) {
    sincospif((float)m / (float)(2 * R.b), &s0, &c0);
  } else {
    sincospif((float)(R.b - m) / (float)(2 * R.b), &c0, &s0);
  }
  float c, s;
  switch (q) {
    case 0: c = c0; s = s0; break;
    case 1: c = -s0; s = c0; break;
    case 2: c = -c0; s = -s0; break;
    default: c = s0; s = -c0; break;
  }
  n[0] = st * c;
  n[1] = st * s;
  n[2] = z;
  return diag;
}

}  // namespace rtg
