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
// Layout for the walk: one 128-byte entry per centre (cx, cy, cz) in
// [1, n]^3, at index ((cz-1) n + (cy-1)) n + (cx-1), holding that
// interpolant's 27 coefficients in powers of f (binary32, computed in FP64
// from the 27 point values): coefficient of fz^k fy^j fx^i at 9k + 3j + i,
// floats 27..31 zero.  Along one axis the quadratic through v(-1), v(0),
// v(1) is v(0) + f (v(1) - v(-1))/2 + f^2 (v(1) - 2 v(0) + v(-1))/2, the same
// polynomial as the three Lagrange weights f(f-1)/2, 1-f^2, f(f+1)/2; so an
// evaluation is one 128-byte line (four 32-byte loads) and 26 FMAs in
// Horner form.
#pragma once
#include "bh_internal.cuh"

namespace bhg {
namespace {

constexpr int kEwaldEntryFloats = 32;

// The grid point c nearest to u/h (s = 2n = 1/h), clamped to [1, n], and
// f = u/h - c.
__device__ __forceinline__ int ewald_axis(float u, float s, int n, float &f) {
  const float t = __fmul_rn(u, s);
  int c = (int)floorf(__fadd_rn(t, 0.5f));
  c = min(max(c, 1), n);
  f = __fsub_rn(t, (float)c);
  return c;
}

// The 128-byte entry of centre (cx, cy, cz), as four 32-byte loads.
__device__ __forceinline__ void ewald_load(const float *tab, int n, int cx, int cy, int cz,
                                           float C[32]) {
  const float *e = tab + (size_t)kEwaldEntryFloats *
                             ((size_t)((cz - 1) * n + (cy - 1)) * n + (cx - 1));
#pragma unroll
  for (int q = 0; q < 4; ++q)
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(C[8 * q]), "=f"(C[8 * q + 1]), "=f"(C[8 * q + 2]), "=f"(C[8 * q + 3]),
          "=f"(C[8 * q + 4]), "=f"(C[8 * q + 5]), "=f"(C[8 * q + 6]), "=f"(C[8 * q + 7])
        : "l"(e + 8 * q));
}

// The interpolant at (fx, fy, fz) from its coefficients, in Horner form:
// x first (9 quadratics), then y (3), then z.
__device__ __forceinline__ float ewald_poly(const float C[32], float fx, float fy, float fz) {
  float px[9];
#pragma unroll
  for (int r = 0; r < 9; ++r)
    px[r] = __fmaf_rn(fx, __fmaf_rn(fx, C[3 * r + 2], C[3 * r + 1]), C[3 * r]);
  float py[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    py[k] = __fmaf_rn(fy, __fmaf_rn(fy, px[3 * k + 2], px[3 * k + 1]), px[3 * k]);
  return __fmaf_rn(fz, __fmaf_rn(fz, py[2], py[1]), py[0]);
}

// chi at |displacement| (ax, ay, az), each >= 0.
__device__ __forceinline__ float ewald_chi(const float *tab, int n, float s, float ax, float ay,
                                           float az) {
  float fx, fy, fz, C[32];
  const int cx = ewald_axis(ax, s, n, fx);
  const int cy = ewald_axis(ay, s, n, fy);
  const int cz = ewald_axis(az, s, n, fz);
  ewald_load(tab, n, cx, cy, cz, C);
  return ewald_poly(C, fx, fy, fz);
}

}  // namespace
}  // namespace bhg
