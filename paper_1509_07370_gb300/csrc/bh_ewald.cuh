// Periodic boundaries (App. A): the table of the Ewald field's smooth part
// and its quadratic interpolation, shared by the table kernels (bh_ewald.cu)
// and the periodic walk (bh_walk_periodic.cu).
//
// psi(r) = 1/|r| + chi(r) is the potential of a unit mass and all its copies
// in the unit-period box, the mean density subtracted; chi is smooth in the
// box around the origin and even in each coordinate.  It is known at the
// points (i, j, k) h, h = 1/(2n), i, j, k = 0 .. n + 1.  At u (per component
// |minimum-image displacement|) each axis takes the point c nearest to u/h,
// clamped to [1, n], and f = u/h - c; the interpolant is the tensor product
// of the three-point quadratics through the points c-1, c, c+1 of each axis.
//
// Layout for the walk: one 64-byte entry per centre (cx, cy, cz) in
// [1, n]^3, at index ((cz-1) n + (cy-1)) n + (cx-1), holding that
// interpolant's 27 coefficients in powers of f, computed in FP64 from the 27
// point values.  Along one axis the quadratic through v(-1), v(0), v(1) is
// v(0) + f (v(1) - v(-1))/2 + f^2 (v(1) - 2 v(0) + v(-1))/2, the same
// polynomial as the three Lagrange weights f(f-1)/2, 1-f^2, f(f+1)/2.  The
// coefficient of fz^k fy^j fx^i is K(k, j, i):
//   bytes  0..15  binary32 K(0,0,0), K(0,0,1), K(0,1,0), K(1,0,0): the value
//                 (about 3) and the first-order terms (up to 0.07 at 32
//                 points per half box);
//   bytes 16..61  binary16, the other 23 in (k, j, i) order: second- and
//                 higher-order terms, at most 2e-3 in size (5.6e-4 at 64
//                 points), so their half-precision rounding changes chi by
//                 less than 3e-7, far below the interpolation error;
//   bytes 62..63  zero.
// A lookup is two 32-byte loads (the L1 data stage, one wavefront per
// distinct line and load, bounds the periodic walk) and 26 FMAs in Horner
// form.
#pragma once
#include <cuda_fp16.h>

#include "bh_internal.cuh"

namespace bhg {
namespace {

constexpr int kEwaldEntryBytes = 64;

// The grid point c nearest to u/h (s = 2n = 1/h), clamped to [1, n], and
// f = u/h - c.
__device__ __forceinline__ int ewald_axis(float u, float s, int n, float &f) {
  const float t = __fmul_rn(u, s);
  int c = (int)floorf(__fadd_rn(t, 0.5f));
  c = min(max(c, 1), n);
  f = __fsub_rn(t, (float)c);
  return c;
}

// Position of K(k, j, i) among the 23 binary16 coefficients (-1: binary32).
// The binary32 ones sit at flat indices 0, 1, 3 and 9 of 9k + 3j + i.
__host__ __device__ constexpr int ewald_half_slot(int k, int j, int i) {
  return (9 * k + 3 * j + i == 0 || 9 * k + 3 * j + i == 1 || 9 * k + 3 * j + i == 3 ||
          9 * k + 3 * j + i == 9)
             ? -1
             : 9 * k + 3 * j + i - (9 * k + 3 * j + i > 9 ? 4 : 9 * k + 3 * j + i > 3 ? 3 : 2);
}

__device__ __forceinline__ float half_lo(uint32_t w) {
  return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
}
__device__ __forceinline__ float half_hi(uint32_t w) {
  return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
}

// The 64-byte entry of centre (cx, cy, cz), as two 32-byte loads (raw words).
__device__ __forceinline__ void ewald_load(const unsigned char *tab, int n, int cx, int cy, int cz,
                                           uint32_t w[16]) {
  const unsigned char *e = tab + (size_t)kEwaldEntryBytes *
                                     (unsigned)(((cz - 1) * n + (cy - 1)) * n + (cx - 1));
#pragma unroll
  for (int q = 0; q < 2; ++q)
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(w[8 * q]), "=r"(w[8 * q + 1]), "=r"(w[8 * q + 2]), "=r"(w[8 * q + 3]),
          "=r"(w[8 * q + 4]), "=r"(w[8 * q + 5]), "=r"(w[8 * q + 6]), "=r"(w[8 * q + 7])
        : "l"(e + 32 * q));
}

// Coefficient K(k, j, i) of an entry, widened to binary32 where it is used.
__device__ __forceinline__ float ewald_coef(const uint32_t w[16], int k, int j, int i) {
  const int f = 9 * k + 3 * j + i;
  if (f == 0) return __uint_as_float(w[0]);
  if (f == 1) return __uint_as_float(w[1]);
  if (f == 3) return __uint_as_float(w[2]);
  if (f == 9) return __uint_as_float(w[3]);
  const int slot = ewald_half_slot(k, j, i);
  return (slot & 1) ? half_hi(w[4 + (slot >> 1)]) : half_lo(w[4 + (slot >> 1)]);
}

// The interpolant at (fx, fy, fz) from an entry, in Horner form: x first (9
// quadratics), then y (3), then z.
__device__ __forceinline__ float ewald_poly(const uint32_t w[16], float fx, float fy, float fz) {
  float px[9];
#pragma unroll
  for (int r = 0; r < 9; ++r)
    px[r] = __fmaf_rn(fx, __fmaf_rn(fx, ewald_coef(w, r / 3, r % 3, 2), ewald_coef(w, r / 3, r % 3, 1)),
                      ewald_coef(w, r / 3, r % 3, 0));
  float py[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    py[k] = __fmaf_rn(fy, __fmaf_rn(fy, px[3 * k + 2], px[3 * k + 1]), px[3 * k]);
  return __fmaf_rn(fz, __fmaf_rn(fz, py[2], py[1]), py[0]);
}

// chi at |displacement| (ax, ay, az), each >= 0.
__device__ __forceinline__ float ewald_chi(const unsigned char *tab, int n, float s, float ax,
                                           float ay, float az) {
  float fx, fy, fz;
  uint32_t w[16];
  const int cx = ewald_axis(ax, s, n, fx);
  const int cy = ewald_axis(ay, s, n, fy);
  const int cz = ewald_axis(az, s, n, fz);
  ewald_load(tab, n, cx, cy, cz, w);
  return ewald_poly(w, fx, fy, fz);
}

}  // namespace
}  // namespace bhg
