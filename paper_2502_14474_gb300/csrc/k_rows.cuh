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

// ---- gathers of the value vector ------------------------------------------
// Global: read-only path (L1/L2).  Ring: a shared-memory window of a banded
// matrix, entry c kept at slot c & mask (see k_bellman.cu, k_gmres.cu).
struct GatherF32 {
  const float* __restrict__ x;
  __device__ __forceinline__ float operator()(int32_t c) const { return __ldg(x + c); }
};
struct RingF32 {
  const float* buf;
  int32_t mask;
  __device__ __forceinline__ float operator()(int32_t c) const { return buf[c & mask]; }
};
struct GatherFF {
  const float2* __restrict__ x;
  __device__ __forceinline__ float2 operator()(int32_t c) const { return __ldg(x + c); }
};
struct RingFF {
  const float2* buf;
  int32_t mask;
  __device__ __forceinline__ float2 operator()(int32_t c) const { return buf[c & mask]; }
};

// ---- FP32 dot: sum val[e] * x[col[e]] over this lane's share of [b, e) -----
template <int VW, typename PV, typename GX>
__device__ __forceinline__ float row_dot_f32(const int32_t* __restrict__ col,
                                             const PV* __restrict__ val, GX x, int64_t b,
                                             int64_t e, int lane, bool vec4) {
  float acc = 0.f;
  if (vec4) {
    const int64_t b4 = (b + 3) & ~int64_t(3);
    const int64_t e4 = e & ~int64_t(3);
    const int64_t hend = b4 < e ? b4 : e;
    for (int64_t i = b + lane; i < hend; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), x(__ldcs(col + i)), acc);
#pragma unroll 2
    for (int64_t i = b4 + 4 * lane; i < e4; i += 4 * VW) {
      const int4 c = __ldcs(reinterpret_cast<const int4*>(col + i));
      const float4 p = Ld<PV>::four(val, i);
      acc = fmaf(p.x, x(c.x), acc);
      acc = fmaf(p.y, x(c.y), acc);
      acc = fmaf(p.z, x(c.z), acc);
      acc = fmaf(p.w, x(c.w), acc);
    }
    const int64_t tb = e4 > b4 ? e4 : b4;
    for (int64_t i = tb + lane; i < e; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), x(__ldcs(col + i)), acc);
  } else {
#pragma unroll 4
    for (int64_t i = b + lane; i < e; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), x(__ldcs(col + i)), acc);
  }
  return acc;
}

// ---- batched rows: RB rows per vector with all loads issued before use ----
// Fast path for matrices whose rows all hold exactly 4*VW entries and start on
// a 16-byte boundary: every lane owns one int4 of col and one 4-entry group of
// val per row, so the loads of RB rows are straight-line and independent.
// Rows with valid[u] == false contribute 0 (their loads are skipped).
template <int VW, int RB, typename PV, typename GX>
__device__ __forceinline__ void rows_dot_f32_k4vw(const int32_t* __restrict__ col,
                                                  const PV* __restrict__ val, GX x,
                                                  const int64_t (&b)[RB], const bool (&valid)[RB],
                                                  int lane, float (&out)[RB]) {
  int4 c[RB];
  float4 p[RB];
#pragma unroll
  for (int u = 0; u < RB; ++u) {
    if (valid[u]) {
      c[u] = __ldcs(reinterpret_cast<const int4*>(col + b[u] + 4 * lane));
      p[u] = Ld<PV>::four(val, b[u] + 4 * lane);
    } else {
      c[u] = make_int4(0, 0, 0, 0);
      p[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
#pragma unroll
  for (int u = 0; u < RB; ++u)
    out[u] = fmaf(p[u].w, x(c[u].w), fmaf(p[u].z, x(c[u].z), fmaf(p[u].y, x(c[u].y),
                                                                   p[u].x * x(c[u].x))));
}

template <int VW, int RB, typename GX>
__device__ __forceinline__ void rows_dot_ff_k4vw(const int32_t* __restrict__ col,
                                                 const float* __restrict__ val, GX V,
                                                 const int64_t (&b)[RB], const bool (&valid)[RB],
                                                 int lane, float (&hi)[RB], float (&lo)[RB]) {
  int4 c[RB];
  float4 p[RB];
#pragma unroll
  for (int u = 0; u < RB; ++u) {
    if (valid[u]) {
      c[u] = __ldcs(reinterpret_cast<const int4*>(col + b[u] + 4 * lane));
      p[u] = __ldcs(reinterpret_cast<const float4*>(val + b[u] + 4 * lane));
    } else {
      c[u] = make_int4(0, 0, 0, 0);
      p[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
#pragma unroll
  for (int u = 0; u < RB; ++u) {
    float h = 0.f, l = 0.f;
    const float2 v0 = V(c[u].x), v1 = V(c[u].y), v2 = V(c[u].z), v3 = V(c[u].w);
    ff_acc(h, l, p[u].x, v0.x, v0.y);
    ff_acc(h, l, p[u].y, v1.x, v1.y);
    ff_acc(h, l, p[u].z, v2.x, v2.y);
    ff_acc(h, l, p[u].w, v3.x, v3.y);
    hi[u] = h;
    lo[u] = l;
  }
}

// Pointer form (global gathers) kept for the callers that stream a vector.
template <int VW, typename PV>
__device__ __forceinline__ float row_dot_f32(const int32_t* __restrict__ col,
                                             const PV* __restrict__ val,
                                             const float* __restrict__ x, int64_t b, int64_t e,
                                             int lane, bool vec4) {
  return row_dot_f32<VW, PV, GatherF32>(col, val, GatherF32{x}, b, e, lane, vec4);
}

// ---- float-float dot over the defining FP32 (+ FP64 remainder) values -------
template <typename GX>
__device__ __forceinline__ void ff_elem(const int32_t* __restrict__ col,
                                        const float* __restrict__ val,
                                        const float* __restrict__ val_lo, GX V, int64_t i,
                                        float& hi, float& lo) {
  const float2 v = V(__ldcs(col + i));
  const float p = __ldcs(val + i);
  ff_acc(hi, lo, p, v.x, v.y);
  if (val_lo) lo = __fmaf_rn(__ldcs(val_lo + i), v.x, lo);
}

template <int VW, typename GX>
__device__ __forceinline__ void row_dot_ff(const int32_t* __restrict__ col,
                                           const float* __restrict__ val,
                                           const float* __restrict__ val_lo, GX V, int64_t b,
                                           int64_t e, int lane, bool vec4, float& hi, float& lo) {
  hi = 0.f;
  lo = 0.f;
  if (vec4 && !val_lo) {
    const int64_t b4 = (b + 3) & ~int64_t(3);
    const int64_t e4 = e & ~int64_t(3);
    const int64_t hend = b4 < e ? b4 : e;
    for (int64_t i = b + lane; i < hend; i += VW) ff_elem(col, val, val_lo, V, i, hi, lo);
#pragma unroll 2
    for (int64_t i = b4 + 4 * lane; i < e4; i += 4 * VW) {
      const int4 c = __ldcs(reinterpret_cast<const int4*>(col + i));
      const float4 p = __ldcs(reinterpret_cast<const float4*>(val + i));
      const float2 v0 = V(c.x), v1 = V(c.y), v2 = V(c.z), v3 = V(c.w);
      ff_acc(hi, lo, p.x, v0.x, v0.y);
      ff_acc(hi, lo, p.y, v1.x, v1.y);
      ff_acc(hi, lo, p.z, v2.x, v2.y);
      ff_acc(hi, lo, p.w, v3.x, v3.y);
    }
    const int64_t tb = e4 > b4 ? e4 : b4;
    for (int64_t i = tb + lane; i < e; i += VW) ff_elem(col, val, val_lo, V, i, hi, lo);
  } else {
#pragma unroll 2
    for (int64_t i = b + lane; i < e; i += VW) ff_elem(col, val, val_lo, V, i, hi, lo);
  }
}

template <int VW>
__device__ __forceinline__ void row_dot_ff(const int32_t* __restrict__ col,
                                           const float* __restrict__ val,
                                           const float* __restrict__ val_lo,
                                           const float2* __restrict__ V, int64_t b, int64_t e,
                                           int lane, bool vec4, float& hi, float& lo) {
  row_dot_ff<VW, GatherFF>(col, val, val_lo, GatherFF{V}, b, e, lane, vec4, hi, lo);
}

}  // namespace mdpk
