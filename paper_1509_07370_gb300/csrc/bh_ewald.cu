// Periodic boundaries (App. A): the Ewald table on the device.
//
// The field is computed once per table (the paper computes it on start-up
// and keeps it in GPU memory for the whole run, App. A and App. B): one
// thread per grid point sums, in FP64,
//   chi(r) =  sum_n' erfc(a |r + n|) / |r + n|  - erf(a |r|) / |r|
//           + (1/pi) sum_{k != 0} exp(-pi^2 |k|^2 / a^2) / |k|^2 cos(2 pi k.r)
//           - pi / a^2
// (n' = every integer triple but 0, components of n and k in [-N, N],
// a = 2, -erf(a r)/r -> -2a/sqrt(pi) at r = 0), i.e. psi(r) - 1/|r|; a second
// kernel turns each centre's 27 neighbouring values into the coefficients of
// the quadratic interpolant the walk evaluates (layout in bh_ewald.cuh).
#include "bh_ewald.cuh"

namespace bhg {
namespace {

constexpr double kEwaldAlpha = 2.0;
constexpr double kPi = 3.14159265358979323846;

__global__ void k_ewald_points(int n, int N, double *__restrict__ chi) {
  const int m = n + 2;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)m * m * m) return;
  const int i = (int)(q % m), j = (int)((q / m) % m), k = (int)(q / ((int64_t)m * m));
  const double h = 0.5 / n;
  const double rx = i * h, ry = j * h, rz = k * h;
  const double a = kEwaldAlpha;
  double real = 0.0;
  for (int i1 = -N; i1 <= N; ++i1)
    for (int i2 = -N; i2 <= N; ++i2)
      for (int i3 = -N; i3 <= N; ++i3) {
        const double x = rx + i1, y = ry + i2, z = rz + i3;
        const double s = sqrt(x * x + y * y + z * z);
        if (i1 == 0 && i2 == 0 && i3 == 0)
          real += s > 0.0 ? -erf(a * s) / s : -2.0 * a / sqrt(kPi);
        else
          real += erfc(a * s) / s;
      }
  double recip = 0.0;
  for (int k1 = -N; k1 <= N; ++k1)
    for (int k2 = -N; k2 <= N; ++k2)
      for (int k3 = -N; k3 <= N; ++k3) {
        if (k1 == 0 && k2 == 0 && k3 == 0) continue;
        const double kk = (double)(k1 * k1 + k2 * k2 + k3 * k3);
        recip += exp(-kPi * kPi * kk / (a * a)) / kk * cospi(2.0 * (k1 * rx + k2 * ry + k3 * rz));
      }
  chi[q] = real + recip / kPi - kPi / (a * a);
}

// Coefficients of the quadratic interpolant around each centre (layout in
// bh_ewald.cuh): the 27 point values, transformed along x, then y, then z by
// [v(-1), v(0), v(1)] -> [v(0), (v(1) - v(-1))/2, (v(1) - 2 v(0) + v(-1))/2],
// in FP64, rounded once to binary32 or binary16 (layout in bh_ewald.cuh).
__global__ void k_ewald_pack(int n, const double *__restrict__ chi,
                             unsigned char *__restrict__ tab) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n * n) return;
  const int m = n + 2;
  const int cx = (int)(e % n) + 1, cy = (int)((e / n) % n) + 1, cz = (int)(e / ((int64_t)n * n)) + 1;
  double v[3][3][3];  // [z][y][x] offsets -1, 0, +1
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a)
        v[c][b][a] = chi[((int64_t)(cz - 1 + c) * m + (cy - 1 + b)) * m + (cx - 1 + a)];
  auto q = [](double &a0, double &a1, double &a2) {
    const double c0 = a1, c1 = 0.5 * (a2 - a0), c2 = 0.5 * (a2 - 2.0 * a1 + a0);
    a0 = c0;
    a1 = c1;
    a2 = c2;
  };
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b) q(v[c][b][0], v[c][b][1], v[c][b][2]);  // along x
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 3; ++a) q(v[c][0][a], v[c][1][a], v[c][2][a]);  // along y
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) q(v[0][b][a], v[1][b][a], v[2][b][a]);  // along z
  unsigned char *out = tab + (int64_t)kEwaldEntryBytes * e;
  float *f32 = reinterpret_cast<float *>(out);
  __half *f16 = reinterpret_cast<__half *>(out + 16);
  f32[0] = (float)v[0][0][0];
  f32[1] = (float)v[0][0][1];
  f32[2] = (float)v[0][1][0];
  f32[3] = (float)v[1][0][0];
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) {
        const int slot = ewald_half_slot(k, j, i);
        if (slot >= 0) f16[slot] = __double2half(v[k][j][i]);
      }
  f16[23] = __ushort_as_half((unsigned short)0);
}

__global__ void k_ewald_eval(int64_t npts, const float *__restrict__ r,
                             const unsigned char *__restrict__ tab, int n,
                             float *__restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npts) return;
  out[q] = ewald_chi(tab, n, (float)(2 * n), fabsf(r[3 * q]), fabsf(r[3 * q + 1]),
                     fabsf(r[3 * q + 2]));
}

}  // namespace

cudaError_t launch_ewald_table(cudaStream_t s, int n, int N, double *scratch,
                               unsigned char *tab) {
  const int m = n + 2;
  const int64_t npts = (int64_t)m * m * m, nent = (int64_t)n * n * n;
  k_ewald_points<<<(unsigned)((npts + 127) / 128), 128, 0, s>>>(n, N, scratch);
  k_ewald_pack<<<(unsigned)((nent + 127) / 128), 128, 0, s>>>(n, scratch, tab);
  return cudaGetLastError();
}

cudaError_t launch_ewald_eval(cudaStream_t s, int64_t npts, const float *r,
                              const unsigned char *tab, int n, float *out) {
  if (npts <= 0) return cudaSuccess;
  k_ewald_eval<<<(unsigned)((npts + 255) / 256), 256, 0, s>>>(npts, r, tab, n, out);
  return cudaGetLastError();
}

}  // namespace bhg
