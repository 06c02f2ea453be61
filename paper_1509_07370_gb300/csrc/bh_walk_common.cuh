// Helpers shared by the walk kernels (bh_walk.cu, bh_walk_learned.cu):
// packed binary32 pair arithmetic and raw record loads in inline PTX, the
// Kahan pair accumulator and the opening-test distance.
#pragma once
#include "bh_internal.cuh"

namespace bhg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
typedef unsigned long long u64;

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// ---- packed binary32 pairs and raw loads (inline PTX) -----------------------
__device__ __forceinline__ u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(u64 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// 1/sqrt(x) on the special-function unit.  Only called where the value is
// used for x >= 2^-44 (an accepted node or another cell), so flushing
// subnormal inputs changes nothing.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// One 32-byte walk record as four 64-bit lanes:
//   q0 = {Px, Px}, q1 = {Py, Pz}, q2 = {M, M}, q3 = {s2, skip}
__device__ __forceinline__ void load_rec(const WalkRec *p, u64 &q0, u64 &q1, u64 &q2, u64 &q3) {
  asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
      : "=l"(q0), "=l"(q1), "=l"(q2), "=l"(q3)
      : "l"(p));
}

// One 32-byte quadrupole record: w0 = {Qxx/2, Qxx/2}, w1 = {Qyy/2, Qzz/2},
// w2 = {Qxy, Qxz}, w3 = {Qyz, 0}.
__device__ __forceinline__ void load_quad(const WalkQuad *p, u64 &w0, u64 &w1, u64 &w2, u64 &w3) {
  asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
      : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
      : "l"(p));
}

// ---- pair walk arithmetic ---------------------------------------------------
// Adds the pair `term` to the running (Kahan-compensated) pair sums.
template <bool KAHAN>
__device__ __forceinline__ void accumulate2(u64 &sum, u64 &comp, u64 term) {
  if (KAHAN) {
    const u64 y = sub2(term, comp);
    const u64 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
  } else {
    sum = add2(sum, term);
  }
}

// Squared distances of the two targets (tx2 = {txa, txb}, ty, tz) to the
// record's binary32 centre of mass, with the fixed rounding of the opening
// test: d2 = fma(dx, dx, fma(dz, dz, dy*dy)); the (dy, dz) part is shared.
__device__ __forceinline__ void dist2(u64 tx2, float ty, float tz, u64 q0, u64 q1, float &d2a,
                                      float &d2b, u64 &dx2, float &dy, float &dz) {
  float py, pz;
  upk(q1, py, pz);
  dx2 = sub2(tx2, q0);
  dy = __fsub_rn(ty, py);
  dz = __fsub_rn(tz, pz);
  const float h = __fmaf_rn(dz, dz, __fmul_rn(dy, dy));
  upk(fma2(dx2, dx2, pk(h, h)), d2a, d2b);
}

}  // namespace
}  // namespace bhg
