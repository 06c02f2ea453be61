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
// The six fields of a walk record (24 bytes: a 128-bit and a 64-bit load)
// as four 64-bit pairs for the packed arithmetic:
//   q0 = {Px, Px}, q1 = {Py, Pz}, q2 = {M, M}, q3 = {s2, skip}
__device__ __forceinline__ void load_rec(const WalkRec *p, u64 &q0, u64 &q1, u64 &q2, u64 &q3) {
  float px, py, pz, m, s2, skf;
  asm("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(px), "=f"(py), "=f"(pz), "=f"(m)
      : "l"(p));
  asm("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(s2), "=f"(skf) : "l"(&p->s2));
  q0 = pk(px, px);
  q1 = pk(py, pz);
  q2 = pk(m, m);
  q3 = pk(s2, skf);
}

// The six fields of a quadrupole record (24 bytes) as w0 = {Qxx/2, Qxx/2},
// w1 = {Qyy/2, Qzz/2}, w2 = {Qxy, Qxz}, w3 = {Qyz, 0}.
__device__ __forceinline__ void load_quad(const WalkQuad *p, u64 &w0, u64 &w1, u64 &w2, u64 &w3) {
  float hxx, hyy, hzz, qxy, qxz, qyz;
  asm("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(hxx), "=f"(hyy), "=f"(hzz), "=f"(qxy)
      : "l"(p));
  asm("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(qxz), "=f"(qyz) : "l"(&p->qxz));
  w0 = pk(hxx, hxx);
  w1 = pk(hyy, hzz);
  w2 = pk(qxy, qxz);
  w3 = pk(qyz, 0.0f);
}

// ---- pair walk arithmetic ---------------------------------------------------
// Compensated summation of the pair `term` into the running pair sums: the
// rounding error of each addition, err = (sum - t) + term with t = sum + term
// (exact while |sum| >= |term|, Fast2Sum), is accumulated apart in `comp`,
// and the result is sum + comp (finish2).  Every term of the walk is
// positive, so the sum grows past each term after the first few.  A zero
// term (a masked target) leaves both exactly unchanged, so the result does
// not depend on which other targets share the warp.
template <bool KAHAN>
__device__ __forceinline__ void accumulate2(u64 &sum, u64 &comp, u64 term) {
  if (KAHAN) {
    const u64 t = add2(sum, term);
    comp = add2(comp, add2(sub2(sum, t), term));
    sum = t;
  } else {
    sum = add2(sum, term);
  }
}
template <bool KAHAN>
__device__ __forceinline__ u64 finish2(u64 sum, u64 comp) {
  return KAHAN ? add2(sum, comp) : sum;
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
