// Row-level building blocks shared by the Bellman and policy-row kernels:
// lane-split dot products of one CSR row with a value vector.
//
// A "vector" is a group of VW consecutive lanes of a warp that together own
// one row.  With vec4 set, the row is split into an unaligned head, a body of
// 16-byte (4-entry) loads of col/val and an unaligned tail, so every HBM
// sector of col/val is read once, coalesced.  col/val/row pointers are
// streamed with evict-first loads (__ldcs) so that the value vector, which is
// gathered, stays resident in L2.
#pragma once

#include "mdp_internal.cuh"

namespace mdpk {

// ---- value loads for the three probability storage types ------------------
template <typename PV>
struct Ld;

template <>
struct Ld<float> {
  static __device__ __forceinline__ float one(const float* p, int64_t i) { return __ldcs(p + i); }
  static __device__ __forceinline__ float4 four(const float* p, int64_t i) {
    return __ldcs(reinterpret_cast<const float4*>(p + i));
  }
};

template <>
struct Ld<__nv_bfloat16> {
  static __device__ __forceinline__ float one(const __nv_bfloat16* p, int64_t i) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p) + i);
    return __uint_as_float(static_cast<unsigned>(u) << 16);
  }
  static __device__ __forceinline__ float4 four(const __nv_bfloat16* p, int64_t i) {
    uint2 u = __ldcs(reinterpret_cast<const uint2*>(p + i));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
  }
};

template <>
struct Ld<__half> {
  static __device__ __forceinline__ float one(const __half* p, int64_t i) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p) + i);
    return __half2float(__ushort_as_half(u));
  }
  static __device__ __forceinline__ float4 four(const __half* p, int64_t i) {
    uint2 u = __ldcs(reinterpret_cast<const uint2*>(p + i));
    float2 a = __half22float2(*reinterpret_cast<__half2*>(&u.x));
    float2 b = __half22float2(*reinterpret_cast<__half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
};

// ---- row bounds ------------------------------------------------------------
template <typename IdxT>
__device__ __forceinline__ void row_bounds(const IdxT* rp, int32_t uniform_len, int64_t r,
                                           int64_t& b, int64_t& e) {
  if (uniform_len > 0) {
    b = r * uniform_len;
    e = b + uniform_len;
  } else {
    b = static_cast<int64_t>(__ldcs(rp + r));
    e = static_cast<int64_t>(__ldcs(rp + r + 1));
  }
}

// ---- FP32 dot: hi += sum val[e] * x[col[e]] over this lane's share ----------
// x is gathered with __ldg (read-only path, L1/L2 resident).
template <int VW, typename PV>
__device__ __forceinline__ float row_dot_f32(const int32_t* __restrict__ col,
                                             const PV* __restrict__ val,
                                             const float* __restrict__ x, int64_t b, int64_t e,
                                             int lane, bool vec4) {
  float acc = 0.f;
  if (vec4) {
    const int64_t b4 = (b + 3) & ~int64_t(3);
    const int64_t e4 = e & ~int64_t(3);
    const int64_t hend = b4 < e ? b4 : e;
    for (int64_t i = b + lane; i < hend; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), __ldg(x + __ldcs(col + i)), acc);
#pragma unroll 2
    for (int64_t i = b4 + 4 * lane; i < e4; i += 4 * VW) {
      const int4 c = __ldcs(reinterpret_cast<const int4*>(col + i));
      const float4 p = Ld<PV>::four(val, i);
      acc = fmaf(p.x, __ldg(x + c.x), acc);
      acc = fmaf(p.y, __ldg(x + c.y), acc);
      acc = fmaf(p.z, __ldg(x + c.z), acc);
      acc = fmaf(p.w, __ldg(x + c.w), acc);
    }
    const int64_t tb = e4 > b4 ? e4 : b4;
    for (int64_t i = tb + lane; i < e; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), __ldg(x + __ldcs(col + i)), acc);
  } else {
#pragma unroll 4
    for (int64_t i = b + lane; i < e; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), __ldg(x + __ldcs(col + i)), acc);
  }
  return acc;
}

// ---- float-float dot over the defining FP32 (+ FP64 remainder) values -------
// V is the float-float vector (x = hi, y = lo).
template <int VW>
__device__ __forceinline__ void ff_elem(const int32_t* __restrict__ col,
                                        const float* __restrict__ val,
                                        const float* __restrict__ val_lo,
                                        const float2* __restrict__ V, int64_t i, float& hi,
                                        float& lo) {
  const float2 v = __ldg(V + __ldcs(col + i));
  const float p = __ldcs(val + i);
  ff_acc(hi, lo, p, v.x, v.y);
  if (val_lo) lo = __fmaf_rn(__ldcs(val_lo + i), v.x, lo);
}

template <int VW>
__device__ __forceinline__ void row_dot_ff(const int32_t* __restrict__ col,
                                           const float* __restrict__ val,
                                           const float* __restrict__ val_lo,
                                           const float2* __restrict__ V, int64_t b, int64_t e,
                                           int lane, bool vec4, float& hi, float& lo) {
  hi = 0.f;
  lo = 0.f;
  if (vec4 && !val_lo) {
    const int64_t b4 = (b + 3) & ~int64_t(3);
    const int64_t e4 = e & ~int64_t(3);
    const int64_t hend = b4 < e ? b4 : e;
    for (int64_t i = b + lane; i < hend; i += VW) ff_elem<VW>(col, val, val_lo, V, i, hi, lo);
#pragma unroll 2
    for (int64_t i = b4 + 4 * lane; i < e4; i += 4 * VW) {
      const int4 c = __ldcs(reinterpret_cast<const int4*>(col + i));
      const float4 p = __ldcs(reinterpret_cast<const float4*>(val + i));
      const float2 v0 = __ldg(V + c.x), v1 = __ldg(V + c.y), v2 = __ldg(V + c.z),
                   v3 = __ldg(V + c.w);
      ff_acc(hi, lo, p.x, v0.x, v0.y);
      ff_acc(hi, lo, p.y, v1.x, v1.y);
      ff_acc(hi, lo, p.z, v2.x, v2.y);
      ff_acc(hi, lo, p.w, v3.x, v3.y);
    }
    const int64_t tb = e4 > b4 ? e4 : b4;
    for (int64_t i = tb + lane; i < e; i += VW) ff_elem<VW>(col, val, val_lo, V, i, hi, lo);
  } else {
#pragma unroll 2
    for (int64_t i = b + lane; i < e; i += VW) ff_elem<VW>(col, val, val_lo, V, i, hi, lo);
  }
}

}  // namespace mdpk
