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

// ---- packed matrix layout ----------------------------------------------------
// The nonzeros are stored in groups of four, each group 32 bytes:
//   [col(4e) col(4e+1) col(4e+2) col(4e+3) | val(4e) .. val(4e+3)]
// over the global entry order (rows are not padded; the last group is).  A row
// of 16 aligned entries is one contiguous 128-byte line, so gathering the rows
// of a policy touches whole lines instead of two half-used ones.  `col` and the
// FP32 `val` below both point at the packed array; these helpers map an entry
// index to its slot.
__device__ __forceinline__ int32_t ldcol(const int32_t* pk, int64_t i) {
  return __ldcs(pk + ((i >> 2) << 3) + (i & 3));
}
// Four columns starting at entry i (i a multiple of 4).
__device__ __forceinline__ int4 ldcol4(const int32_t* pk, int64_t i) {
  return __ldcs(reinterpret_cast<const int4*>(pk + 2 * i));
}

// ---- value loads for the three probability storage types ------------------
template <typename PV>
struct Ld;

template <>
struct Ld<float> {  // FP32 values live in the packed array
  static __device__ __forceinline__ float one(const float* pk, int64_t i) {
    return __ldcs(pk + ((i >> 2) << 3) + 4 + (i & 3));
  }
  static __device__ __forceinline__ float4 four(const float* pk, int64_t i) {
    return __ldcs(reinterpret_cast<const float4*>(pk + 2 * i + 4));
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

// ---- one thread per row, whole packed groups --------------------------------
// For short or unaligned rows: the thread loads every 4-entry group that
// overlaps [b, e) with one int4 of columns and one 4-value load, and adds the
// entries inside the row strictly in entry order (so identical rows give
// identical sums whatever their alignment).  Entries outside the row are not
// gathered.  The value array must be padded to a multiple of 4 entries.
template <typename PV, typename GX>
__device__ __forceinline__ float row_dot_f32_g1(const int32_t* __restrict__ col,
                                                const PV* __restrict__ val, GX x, int64_t b,
                                                int64_t e) {
  float acc = 0.f;
  const int64_t g1 = (e + 3) >> 2;
#pragma unroll 2
  for (int64_t g = b >> 2; g < g1; ++g) {
    const int64_t i0 = g << 2;
    const int4 c = ldcol4(col, i0);
    const float4 p = Ld<PV>::four(val, i0);
    if (i0 >= b) acc = fmaf(p.x, x(c.x), acc);
    if (i0 + 1 >= b && i0 + 1 < e) acc = fmaf(p.y, x(c.y), acc);
    if (i0 + 2 >= b && i0 + 2 < e) acc = fmaf(p.z, x(c.z), acc);
    if (i0 + 3 >= b && i0 + 3 < e) acc = fmaf(p.w, x(c.w), acc);
  }
  return acc;
}

// Short row with its first two packed groups loaded ahead: `row_pre` issues
// the loads, `row_pre_dot` adds the entries of [b, e) in entry order (the
// prefetched groups first, then any further groups), so several rows of one
// thread can have their loads in flight together.
template <typename PV>
struct RowPre {
  int4 c0, c1;
  float4 v0, v1;
  int64_t b, e;
};

template <typename PV>
__device__ __forceinline__ void row_pre(const int32_t* __restrict__ col, const PV* __restrict__ val,
                                        int64_t b, int64_t e, RowPre<PV>& R) {
  R.b = b;
  R.e = e;
  const int64_t i0 = (b >> 2) << 2;
  R.c0 = make_int4(0, 0, 0, 0);
  R.c1 = R.c0;
  R.v0 = make_float4(0.f, 0.f, 0.f, 0.f);
  R.v1 = R.v0;
  if (i0 < e) {
    R.c0 = ldcol4(col, i0);
    R.v0 = Ld<PV>::four(val, i0);
  }
  if (i0 + 4 < e) {
    R.c1 = ldcol4(col, i0 + 4);
    R.v1 = Ld<PV>::four(val, i0 + 4);
  }
}

template <typename PV, typename GX>
__device__ __forceinline__ float row_pre_dot(const int32_t* __restrict__ col,
                                             const PV* __restrict__ val, GX x, const RowPre<PV>& R) {
  const int64_t b = R.b, e = R.e;
  const int64_t i0 = (b >> 2) << 2;
  float acc = 0.f;
  const int cc[8] = {R.c0.x, R.c0.y, R.c0.z, R.c0.w, R.c1.x, R.c1.y, R.c1.z, R.c1.w};
  const float pp[8] = {R.v0.x, R.v0.y, R.v0.z, R.v0.w, R.v1.x, R.v1.y, R.v1.z, R.v1.w};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t i = i0 + q;
    if (i >= b && i < e) acc = fmaf(pp[q], x(cc[q]), acc);
  }
  for (int64_t g = (i0 >> 2) + 2; (g << 2) < e; ++g) {
    const int64_t j0 = g << 2;
    const int4 c = ldcol4(col, j0);
    const float4 p = Ld<PV>::four(val, j0);
    acc = fmaf(p.x, x(c.x), acc);
    if (j0 + 1 < e) acc = fmaf(p.y, x(c.y), acc);
    if (j0 + 2 < e) acc = fmaf(p.z, x(c.z), acc);
    if (j0 + 3 < e) acc = fmaf(p.w, x(c.w), acc);
  }
  return acc;
}

// Float-float form of row_pre_dot over rows prefetched by row_pre (FP32
// values, no FP64 low parts): the same entries in the same order as
// row_dot_ff_g1, so the sums are bitwise those of row_dot_ff_g1.
template <typename GX>
__device__ __forceinline__ void row_pre_dot_ff(const int32_t* __restrict__ col,
                                               const float* __restrict__ val, GX V,
                                               const RowPre<float>& R, float& hi, float& lo) {
  hi = 0.f;
  lo = 0.f;
  const int64_t b = R.b, e = R.e;
  const int64_t i0 = (b >> 2) << 2;
  const int cc[8] = {R.c0.x, R.c0.y, R.c0.z, R.c0.w, R.c1.x, R.c1.y, R.c1.z, R.c1.w};
  const float pp[8] = {R.v0.x, R.v0.y, R.v0.z, R.v0.w, R.v1.x, R.v1.y, R.v1.z, R.v1.w};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t i = i0 + q;
    if (i >= b && i < e) {
      const float2 v = V(cc[q]);
      ff_acc(hi, lo, pp[q], v.x, v.y);
    }
  }
  for (int64_t g = (i0 >> 2) + 2; (g << 2) < e; ++g) {
    const int64_t j0 = g << 2;
    const int4 c = ldcol4(col, j0);
    const float4 p = Ld<float>::four(val, j0);
    const int cq[4] = {c.x, c.y, c.z, c.w};
    const float pq[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (j0 + q < e) {
        const float2 v = V(cq[q]);
        ff_acc(hi, lo, pq[q], v.x, v.y);
      }
    }
  }
}

template <typename GX>
__device__ __forceinline__ void row_dot_ff_g1(const int32_t* __restrict__ col,
                                              const float* __restrict__ val,
                                              const float* __restrict__ val_lo, GX V, int64_t b,
                                              int64_t e, float& hi, float& lo) {
  hi = 0.f;
  lo = 0.f;
  const int64_t g1 = (e + 3) >> 2;
#pragma unroll 2
  for (int64_t g = b >> 2; g < g1; ++g) {
    const int64_t i0 = g << 2;
    const int4 c = ldcol4(col, i0);
    const float4 p = Ld<float>::four(val, i0);
    const int cc[4] = {c.x, c.y, c.z, c.w};
    const float pp[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + q;
      if (i >= b && i < e) {
        const float2 v = V(cc[q]);
        ff_acc(hi, lo, pp[q], v.x, v.y);
        if (val_lo) lo = __fmaf_rn(__ldcs(val_lo + i), v.x, lo);
      }
    }
  }
}

// ---- FP32 dot: sum val[e] * x[col[e]] over this lane's share of [b, e) -----
template <int VW, typename PV, typename GX>
__device__ __forceinline__ float row_dot_f32(const int32_t* __restrict__ col,
                                             const PV* __restrict__ val, GX x, int64_t b,
                                             int64_t e, int lane, bool vec4) {
  if constexpr (VW == 1) return row_dot_f32_g1<PV, GX>(col, val, x, b, e);
  float acc = 0.f;
  if (vec4) {
    const int64_t b4 = (b + 3) & ~int64_t(3);
    const int64_t e4 = e & ~int64_t(3);
    const int64_t hend = b4 < e ? b4 : e;
    for (int64_t i = b + lane; i < hend; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), x(ldcol(col, i)), acc);
#pragma unroll 2
    for (int64_t i = b4 + 4 * lane; i < e4; i += 4 * VW) {
      const int4 c = ldcol4(col, i);
      const float4 p = Ld<PV>::four(val, i);
      acc = fmaf(p.x, x(c.x), acc);
      acc = fmaf(p.y, x(c.y), acc);
      acc = fmaf(p.z, x(c.z), acc);
      acc = fmaf(p.w, x(c.w), acc);
    }
    const int64_t tb = e4 > b4 ? e4 : b4;
    for (int64_t i = tb + lane; i < e; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), x(ldcol(col, i)), acc);
  } else {
#pragma unroll 4
    for (int64_t i = b + lane; i < e; i += VW)
      acc = fmaf(Ld<PV>::one(val, i), x(ldcol(col, i)), acc);
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
      c[u] = ldcol4(col, b[u] + 4 * lane);
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
      c[u] = ldcol4(col, b[u] + 4 * lane);
      p[u] = Ld<float>::four(val, b[u] + 4 * lane);
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

// ---- reduce-scatter across the VW lanes of a vector -------------------------
// On entry lane l holds its partial sums p[u] of the vector's rows u < VW; on
// exit the return value of lane l is the full sum of row l.  The association
// is the same for every row ((x0 + x2) + (x1 + x3) for VW = 4), so rows with
// identical entries give identical sums.
template <int VW>
__device__ __forceinline__ float reduce_scatter(const float (&p)[VW], int lane);

template <>
__device__ __forceinline__ float reduce_scatter<1>(const float (&p)[1], int) {
  return p[0];
}

template <>
__device__ __forceinline__ float reduce_scatter<2>(const float (&p)[2], int lane) {
  const bool up = lane & 1;
  const float keep = up ? p[1] : p[0];
  const float send = up ? p[0] : p[1];
  return keep + __shfl_xor_sync(0xffffffffu, send, 1);
}

template <>
__device__ __forceinline__ float reduce_scatter<4>(const float (&p)[4], int lane) {
  const bool up2 = lane & 2;
  float k0 = up2 ? p[2] : p[0], k1 = up2 ? p[3] : p[1];
  const float s0 = up2 ? p[0] : p[2], s1 = up2 ? p[1] : p[3];
  k0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  const bool up1 = lane & 1;
  const float keep = up1 ? k1 : k0;
  const float send = up1 ? k0 : k1;
  return keep + __shfl_xor_sync(0xffffffffu, send, 1);
}

// Float-float version: (hi, lo) pairs combined with TwoSum on the high parts.
__device__ __forceinline__ void ff_merge(float& hi, float& lo, float ohi, float olo) {
  float s, e;
  two_sum(hi, ohi, s, e);
  hi = s;
  lo = __fadd_rn(__fadd_rn(lo, olo), e);
}

template <int VW>
__device__ __forceinline__ void reduce_scatter_ff(const float (&ph)[VW], const float (&pl)[VW],
                                                  int lane, float& hi, float& lo);

template <>
__device__ __forceinline__ void reduce_scatter_ff<1>(const float (&ph)[1], const float (&pl)[1],
                                                     int, float& hi, float& lo) {
  hi = ph[0];
  lo = pl[0];
}

template <>
__device__ __forceinline__ void reduce_scatter_ff<2>(const float (&ph)[2], const float (&pl)[2],
                                                     int lane, float& hi, float& lo) {
  const bool up = lane & 1;
  hi = up ? ph[1] : ph[0];
  lo = up ? pl[1] : pl[0];
  const float sh = up ? ph[0] : ph[1], sl = up ? pl[0] : pl[1];
  ff_merge(hi, lo, __shfl_xor_sync(0xffffffffu, sh, 1), __shfl_xor_sync(0xffffffffu, sl, 1));
}

template <>
__device__ __forceinline__ void reduce_scatter_ff<4>(const float (&ph)[4], const float (&pl)[4],
                                                     int lane, float& hi, float& lo) {
  const bool up2 = lane & 2;
  float k0h = up2 ? ph[2] : ph[0], k0l = up2 ? pl[2] : pl[0];
  float k1h = up2 ? ph[3] : ph[1], k1l = up2 ? pl[3] : pl[1];
  const float s0h = up2 ? ph[0] : ph[2], s0l = up2 ? pl[0] : pl[2];
  const float s1h = up2 ? ph[1] : ph[3], s1l = up2 ? pl[1] : pl[3];
  ff_merge(k0h, k0l, __shfl_xor_sync(0xffffffffu, s0h, 2), __shfl_xor_sync(0xffffffffu, s0l, 2));
  ff_merge(k1h, k1l, __shfl_xor_sync(0xffffffffu, s1h, 2), __shfl_xor_sync(0xffffffffu, s1l, 2));
  const bool up1 = lane & 1;
  hi = up1 ? k1h : k0h;
  lo = up1 ? k1l : k0l;
  const float sh = up1 ? k0h : k1h, sl = up1 ? k0l : k1l;
  ff_merge(hi, lo, __shfl_xor_sync(0xffffffffu, sh, 1), __shfl_xor_sync(0xffffffffu, sl, 1));
}

// ---- VW rows per vector, 4*VW entries per row (uniform, 16-byte aligned) ---
// Lane l loads entries [4l, 4l+4) of each of the vector's VW rows (row u starts
// at b[u]); the loads of all rows are issued before any gather.  Rows with
// valid[u] false contribute 0.  Returns lane l's partial sums p[u].
template <int VW, typename PV, typename GX>
__device__ __forceinline__ void vec_rows_f32(const int32_t* __restrict__ col,
                                             const PV* __restrict__ val, GX x,
                                             const int64_t (&b)[VW], const bool (&valid)[VW],
                                             int lane, float (&p)[VW]) {
  int4 c[VW];
  float4 q[VW];
#pragma unroll
  for (int u = 0; u < VW; ++u) {
    if (valid[u]) {
      c[u] = ldcol4(col, b[u] + 4 * lane);
      q[u] = Ld<PV>::four(val, b[u] + 4 * lane);
    } else {
      c[u] = make_int4(0, 0, 0, 0);
      q[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
#pragma unroll
  for (int u = 0; u < VW; ++u)
    p[u] = fmaf(q[u].w, x(c[u].w), fmaf(q[u].z, x(c[u].z), fmaf(q[u].y, x(c[u].y),
                                                                 q[u].x * x(c[u].x))));
}

// ff_acc on two independent sums at once with the packed FP32x2 instructions:
// each lane of the pair goes through exactly the operations of ff_acc, so the
// results are bitwise those of two scalar calls.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void ff_acc2(float2& s_hi, float2& s_lo, float2 p, float2 vhi,
                                        float2 vlo) {
  const float2 ph = __fmul2_rn(p, vhi);
  float2 pl = __ffma2_rn(p, vhi, neg2(ph));
  pl = __ffma2_rn(p, vlo, pl);
  const float2 t = __fadd2_rn(s_hi, ph);
  const float2 bb = __fadd2_rn(t, neg2(s_hi));
  const float2 e = __fadd2_rn(__fadd2_rn(s_hi, neg2(__fadd2_rn(t, neg2(bb)))),
                              __fadd2_rn(ph, neg2(bb)));
  s_hi = t;
  s_lo = __fadd2_rn(s_lo, __fadd2_rn(e, pl));
}

template <int VW, typename GX>
__device__ __forceinline__ void vec_rows_ff(const int32_t* __restrict__ col,
                                            const float* __restrict__ val, GX V,
                                            const int64_t (&b)[VW], const bool (&valid)[VW],
                                            int lane, float (&ph)[VW], float (&pl)[VW]) {
  int4 c[VW];
  float4 q[VW];
#pragma unroll
  for (int u = 0; u < VW; ++u) {
    if (valid[u]) {
      c[u] = ldcol4(col, b[u] + 4 * lane);
      q[u] = Ld<float>::four(val, b[u] + 4 * lane);
    } else {
      c[u] = make_int4(0, 0, 0, 0);
      q[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if constexpr (VW % 2 == 0) {
    // rows u and u + 1 side by side in the packed instructions
#pragma unroll
    for (int u = 0; u < VW; u += 2) {
      float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
      const float2 a0 = V(c[u].x), a1 = V(c[u].y), a2 = V(c[u].z), a3 = V(c[u].w);
      const float2 b0 = V(c[u + 1].x), b1 = V(c[u + 1].y), b2 = V(c[u + 1].z),
                   b3 = V(c[u + 1].w);
      ff_acc2(h, l, make_float2(q[u].x, q[u + 1].x), make_float2(a0.x, b0.x),
              make_float2(a0.y, b0.y));
      ff_acc2(h, l, make_float2(q[u].y, q[u + 1].y), make_float2(a1.x, b1.x),
              make_float2(a1.y, b1.y));
      ff_acc2(h, l, make_float2(q[u].z, q[u + 1].z), make_float2(a2.x, b2.x),
              make_float2(a2.y, b2.y));
      ff_acc2(h, l, make_float2(q[u].w, q[u + 1].w), make_float2(a3.x, b3.x),
              make_float2(a3.y, b3.y));
      ph[u] = h.x;
      pl[u] = l.x;
      ph[u + 1] = h.y;
      pl[u + 1] = l.y;
    }
  } else {
#pragma unroll
    for (int u = 0; u < VW; ++u) {
      float h = 0.f, l = 0.f;
      const float2 v0 = V(c[u].x), v1 = V(c[u].y), v2 = V(c[u].z), v3 = V(c[u].w);
      ff_acc(h, l, q[u].x, v0.x, v0.y);
      ff_acc(h, l, q[u].y, v1.x, v1.y);
      ff_acc(h, l, q[u].z, v2.x, v2.y);
      ff_acc(h, l, q[u].w, v3.x, v3.y);
      ph[u] = h;
      pl[u] = l;
    }
  }
}

// ---- packed 16-bit inner copy ------------------------------------------------
// Group g is one uint4: .x/.y hold int16 offsets (col - s) of entries 4g..4g+3
// from the state s of the entry's row, .z/.w the 16-bit values.  A policy row
// of 16 entries is 64 bytes (half the FP32 group bytes).
template <typename Q>
struct Q16;
template <>
struct Q16<__nv_bfloat16> {
  static __device__ __forceinline__ float f(uint32_t u) { return __uint_as_float(u << 16); }
};
template <>
struct Q16<__half> {
  static __device__ __forceinline__ float f(uint32_t u) {
    return __half2float(__ushort_as_half(static_cast<unsigned short>(u & 0xffffu)));
  }
};

__device__ __forceinline__ int32_t lp_off(uint32_t w, int hi) {
  return static_cast<int32_t>(static_cast<int16_t>(hi ? (w >> 16) : (w & 0xffffu)));
}

// Entries of group G (entry indices i0..i0+3) that fall inside [b, e), in
// order: num += q_e x(col_e), den += q_e.  The row's renormalised inner
// operator is num / den (row sum of the rounded values computed on the fly,
// so no per-row factor has to be gathered).
template <typename Q, typename GX>
__device__ __forceinline__ void lp_group_dot(uint4 G, int64_t i0, int64_t b, int64_t e, int64_t s,
                                             GX x, float& num, float& den) {
  const uint32_t dw[2] = {G.x, G.y};
  const uint32_t qw[2] = {G.z, G.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t i = i0 + q;
    if (i >= b && i < e) {
      const int32_t c = static_cast<int32_t>(s) + lp_off(dw[q >> 1], q & 1);
      const float v = Q16<Q>::f(q & 1 ? (qw[q >> 1] >> 16) : (qw[q >> 1] & 0xffffu));
      num = fmaf(v, x(c), num);
      den += v;
    }
  }
}

// The same over the entries q of group G with lo <= q < hi (positions
// relative to the group's first entry; 32-bit bounds for short rows).
template <typename Q, typename GX>
__device__ __forceinline__ void lp_group_dot_rel(uint4 G, int32_t lo, int32_t hi, int64_t s, GX x,
                                                 float& num, float& den) {
  const uint32_t dw[2] = {G.x, G.y};
  const uint32_t qw[2] = {G.z, G.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q >= lo && q < hi) {
      const int32_t c = static_cast<int32_t>(s) + lp_off(dw[q >> 1], q & 1);
      const float v = Q16<Q>::f(q & 1 ? (qw[q >> 1] >> 16) : (qw[q >> 1] & 0xffffu));
      num = fmaf(v, x(c), num);
      den += v;
    }
  }
}

// Lane `lane` of VW takes groups g0 + lane, g0 + lane + VW, ... of row [b, e)
// of state s; the caller reduces num and den over the VW lanes.
template <int VW, typename Q, typename GX>
__device__ __forceinline__ void row_dot_lp(const uint4* __restrict__ lpk, GX x, int64_t s,
                                           int64_t b, int64_t e, int lane, float& num,
                                           float& den) {
  num = 0.f;
  den = 0.f;
  const int64_t g1 = (e + 3) >> 2;
#pragma unroll 2
  for (int64_t g = (b >> 2) + lane; g < g1; g += VW)
    lp_group_dot<Q>(__ldcs(lpk + g), g << 2, b, e, s, x, num, den);
}

// Fast path: VW rows (states srow[u]) of 4*VW aligned entries; lane l loads
// group l of each row before any gather.
template <int VW, typename Q, typename GX>
__device__ __forceinline__ void vec_rows_lp(const uint4* __restrict__ lpk, GX x,
                                            const int64_t (&b)[VW], const int64_t (&srow)[VW],
                                            const bool (&valid)[VW], int lane, float (&num)[VW],
                                            float (&den)[VW]) {
  uint4 G[VW];
#pragma unroll
  for (int u = 0; u < VW; ++u)
    G[u] = valid[u] ? __ldcs(lpk + (b[u] >> 2) + lane) : make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int u = 0; u < VW; ++u) {
    const int64_t i0 = b[u] + 4 * lane;
    num[u] = 0.f;
    den[u] = 0.f;
    if (valid[u]) lp_group_dot<Q>(G[u], i0, i0, i0 + 4, srow[u], x, num[u], den[u]);
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
  const float2 v = V(ldcol(col, i));
  const float p = Ld<float>::one(val, i);
  ff_acc(hi, lo, p, v.x, v.y);
  if (val_lo) lo = __fmaf_rn(__ldcs(val_lo + i), v.x, lo);
}

template <int VW, typename GX>
__device__ __forceinline__ void row_dot_ff(const int32_t* __restrict__ col,
                                           const float* __restrict__ val,
                                           const float* __restrict__ val_lo, GX V, int64_t b,
                                           int64_t e, int lane, bool vec4, float& hi, float& lo) {
  if constexpr (VW == 1) {
    row_dot_ff_g1<GX>(col, val, val_lo, V, b, e, hi, lo);
    return;
  }
  hi = 0.f;
  lo = 0.f;
  if (vec4 && !val_lo) {
    const int64_t b4 = (b + 3) & ~int64_t(3);
    const int64_t e4 = e & ~int64_t(3);
    const int64_t hend = b4 < e ? b4 : e;
    for (int64_t i = b + lane; i < hend; i += VW) ff_elem(col, val, val_lo, V, i, hi, lo);
#pragma unroll 2
    for (int64_t i = b4 + 4 * lane; i < e4; i += 4 * VW) {
      const int4 c = ldcol4(col, i);
      const float4 p = Ld<float>::four(val, i);
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
