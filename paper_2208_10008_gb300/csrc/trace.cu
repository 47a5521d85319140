// Ray traversal (Sec. III.B, Fig. 4 of arXiv 2208.10008): collision detection
// of a ray with the BVH -- test the bounding boxes, descend into the ones the
// ray meets, test the triangles of the leaves reached and keep the nearest hit.
//
// k_trace (float32, one ray per thread)
//   * 4-wide nodes, one 128-byte line each, read with 16-byte read-only loads;
//     children ordered near-first on a per-thread stack.
//   * box test: slab test with the near/far plane picked by the sign of 1/d
//     (NaN-safe for axis-parallel rays); the interval is widened by a relative
//     1e-6 so rounding never drops a box the exact ray meets.
//   * ray action range: boxes are culled beyond min(tmax, best t + window),
//     so the ray's maximal range bounds the walk (abstract, Sec. II.B).
//   * triangle test: the watertight test of Woop, Benthin and Wald (JCGT
//     2013), two-sided, plus a forward error bound E on its three edge
//     functions.  Signs settled beyond E give a certain hit or miss; anything
//     else, a second hit within the error window of the best one, a hit near
//     tmin / tmax, or a stack overflow marks the ray for k_retest64.
// k_retest64 (float64, flagged rays only)
//   * rays with a candidate list: a group of lanes per ray (a warp when few
//     rays are flagged, one lane when many are) applies the float64 rule to
//     the candidates and a group reduction keeps the nearest; when the
//     list overflowed, one thread per ray does a stackless walk of the
//     binary tree (parent links) with the same conservative float32 box test
//     culled at the float64 best distance, and for every triangle the
//     float32 bound does not prove missed, the reference hit rule:
//     Moller-Trumbore with inclusive edges, |det| <= 1e-14 |e1||e2||d| is
//     parallel, tmin < t < tmax, lowest id on equal t, with the operation
//     order fixed and no contraction, so its answer is the float64
//     definition's answer bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kTraceBlock = 128;
constexpr int kStack = 64;  // default depth of the walk's stack
constexpr int kRetestBlock = 128;
constexpr unsigned kFullMask = 0xffffffffu;
constexpr float kU = 5.9604645e-08f;   // unit roundoff of float32, 2^-24
constexpr float kWiden = 1e-6f;        // relative widening of box intervals
constexpr float kTieRel = 1e-5f;       // relative window of the best-hit checks
constexpr int kCand = kTraceCand;      // float64 candidates remembered per ray

struct RayPre {
  float ox, oy, oz, tmin, tmax;
  float ix, iy, iz;  // 1/d
  int sx, sy, sz;    // 1 when the axis runs negative: the near plane is the box's hi
  float Sx, Sy, Sz;  // shear constants of the watertight test
  int kx, ky, kz;
  bool valid;
};

__device__ __forceinline__ float sel3(float x, float y, float z, int k) {
  return k == 0 ? x : (k == 1 ? y : z);
}

__device__ __forceinline__ RayPre setup_ray(float4 a, float4 b) {
  RayPre r;
  r.ox = a.x;
  r.oy = a.y;
  r.oz = a.z;
  r.tmin = a.w;
  r.tmax = b.w;
  float dx = b.x, dy = b.y, dz = b.z;
  bool fin = isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(dx) && isfinite(dy) &&
             isfinite(dz) && !isnan(a.w) && !isnan(b.w);
  r.valid = fin && (b.w > a.w) && (dx != 0.f || dy != 0.f || dz != 0.f);
  r.ix = __frcp_rn(dx);
  r.iy = __frcp_rn(dy);
  r.iz = __frcp_rn(dz);
  r.sx = r.ix >= 0.f ? 0 : 1;
  r.sy = r.iy >= 0.f ? 0 : 1;
  r.sz = r.iz >= 0.f ? 0 : 1;
  float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
  int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  float dkz = sel3(dx, dy, dz, kz);
  if (dkz < 0.f) {
    int t = kx;
    kx = ky;
    ky = t;
  }
  r.kx = kx;
  r.ky = ky;
  r.kz = kz;
  r.Sx = __fdiv_rn(sel3(dx, dy, dz, kx), dkz);
  r.Sy = __fdiv_rn(sel3(dx, dy, dz, ky), dkz);
  r.Sz = __frcp_rn(dkz);
  return r;
}

// Watertight test with a forward error bound.  cls: 0 certain miss,
// 1 certain hit (t, errT, u, v valid), 2 uncertain (tlo..thi brackets any t).
struct TriRes {
  int cls;
  float t, err, u, v, tlo, thi;
};

__device__ __forceinline__ TriRes tri_test(const RayPre& r, float4 a, float4 b, float4 c) {
  TriRes res;
  float Ax0 = __fsub_rn(a.x, r.ox), Ay0 = __fsub_rn(a.y, r.oy), Az0 = __fsub_rn(a.z, r.oz);
  float Bx0 = __fsub_rn(b.x, r.ox), By0 = __fsub_rn(b.y, r.oy), Bz0 = __fsub_rn(b.z, r.oz);
  float Cx0 = __fsub_rn(c.x, r.ox), Cy0 = __fsub_rn(c.y, r.oy), Cz0 = __fsub_rn(c.z, r.oz);
  float Akz = sel3(Ax0, Ay0, Az0, r.kz), Bkz = sel3(Bx0, By0, Bz0, r.kz), Ckz = sel3(Cx0, Cy0, Cz0, r.kz);
  float Ax = __fmaf_rn(-r.Sx, Akz, sel3(Ax0, Ay0, Az0, r.kx));
  float Ay = __fmaf_rn(-r.Sy, Akz, sel3(Ax0, Ay0, Az0, r.ky));
  float Bx = __fmaf_rn(-r.Sx, Bkz, sel3(Bx0, By0, Bz0, r.kx));
  float By = __fmaf_rn(-r.Sy, Bkz, sel3(Bx0, By0, Bz0, r.ky));
  float Cx = __fmaf_rn(-r.Sx, Ckz, sel3(Cx0, Cy0, Cz0, r.kx));
  float Cy = __fmaf_rn(-r.Sy, Ckz, sel3(Cx0, Cy0, Cz0, r.ky));
  float U = __fmaf_rn(Cx, By, -__fmul_rn(Cy, Bx));
  float V = __fmaf_rn(Ax, Cy, -__fmul_rn(Ay, Cx));
  float W = __fmaf_rn(Bx, Ay, -__fmul_rn(By, Ax));
  // Forward error bound of U, V, W against exact arithmetic on the same
  // float32 inputs: |dU| <= u P (12 R + 7 P) with R the largest translated
  // coordinate and P the largest projected one (13 R + 8 P keeps a margin).
  float R = fmaxf(fmaxf(fmaxf(fabsf(Ax0), fabsf(Ay0)), fmaxf(fabsf(Az0), fabsf(Bx0))),
                  fmaxf(fmaxf(fabsf(By0), fabsf(Bz0)), fmaxf(fmaxf(fabsf(Cx0), fabsf(Cy0)), fabsf(Cz0))));
  float P = fmaxf(fmaxf(fmaxf(fabsf(Ax), fabsf(Ay)), fmaxf(fabsf(Bx), fabsf(By))),
                  fmaxf(fabsf(Cx), fabsf(Cy)));
  float E = kU * P * (13.f * R + 8.f * P);
  float mn = fminf(U, fminf(V, W)), mx = fmaxf(U, fmaxf(V, W));
  float Zs = fabsf(r.Sz);
  float Az = __fmul_rn(r.Sz, Akz), Bz = __fmul_rn(r.Sz, Bkz), Cz = __fmul_rn(r.Sz, Ckz);
  if (mn < -E && mx > E) {
    res.cls = 0;
    return res;
  }
  if (mn > E || mx < -E) {
    float det = __fadd_rn(__fadd_rn(U, V), W);
    float T = __fmaf_rn(U, Az, __fmaf_rn(V, Bz, __fmul_rn(W, Cz)));
    float t = __fdiv_rn(T, det);
    float zs = fmaxf(fmaxf(fabsf(Az - t), fabsf(Bz - t)), fabsf(Cz - t));
    res.cls = 1;
    res.t = t;
    res.err = 3.01f * E * zs / fabsf(det) + 8.f * kU * Zs * R;
    float id = __frcp_rn(det);
    res.u = V * id;
    res.v = W * id;
    return res;
  }
  // uncertain: any hit lies between the smallest and largest vertex depth
  float slack = 4.f * kU * Zs * R;
  res.cls = 2;
  res.tlo = fminf(Az, fminf(Bz, Cz)) - slack;
  res.thi = fmaxf(Az, fmaxf(Bz, Cz)) + slack;
  return res;
}

// ---------------------------------------------------------------- float-float
// Double-float arithmetic from error-free transformations: TwoSum (Knuth),
// TwoProduct with a fused multiply-add, and the usual renormalisation
// (Dekker 1971).  Used once per ray to recompute the distance of the chosen
// hit when its float32 error bound is not already inside the tolerance.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  float e = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, e);
  e = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return quick_two_sum(p, e);
}

// Distance along the ray to the plane of (v0, v1, v2):
// t = n.(v0 - o) / n.d with n = (v1 - v0) x (v2 - v0), all in float-float
// (the differences are exact), rounded once to float at the end.
__device__ float refine_t(const RayPre& r, float dx, float dy, float dz, float4 a, float4 b, float4 c) {
  ff Ax = two_sum(a.x, -r.ox), Ay = two_sum(a.y, -r.oy), Az = two_sum(a.z, -r.oz);
  ff e1x = two_sum(b.x, -a.x), e1y = two_sum(b.y, -a.y), e1z = two_sum(b.z, -a.z);
  ff e2x = two_sum(c.x, -a.x), e2y = two_sum(c.y, -a.y), e2z = two_sum(c.z, -a.z);
  ff nx = ff_add(ff_mul(e1y, e2z), ff_neg(ff_mul(e1z, e2y)));
  ff ny = ff_add(ff_mul(e1z, e2x), ff_neg(ff_mul(e1x, e2z)));
  ff nz = ff_add(ff_mul(e1x, e2y), ff_neg(ff_mul(e1y, e2x)));
  ff num = ff_add(ff_add(ff_mul(nx, Ax), ff_mul(ny, Ay)), ff_mul(nz, Az));
  ff den = ff_add(ff_add(ff_mulf(nx, dx), ff_mulf(ny, dy)), ff_mulf(nz, dz));
  float q = __fdiv_rn(num.hi, den.hi);
  ff rem = ff_add(num, ff_neg(ff_mulf(den, q)));
  return __fadd_rn(q, __fdiv_rn(rem.hi, den.hi));
}

// Slab test of the 4 children of a node; returns a bit mask of children
// whose widened interval meets [tmin, bound], near distances in tn[].
__device__ __forceinline__ unsigned slab4(const WNode* __restrict__ node, const RayPre& r, float bound,
                                          float tn[4], int4* child) {
  // planes lo x, hi x, lo y, hi y, lo z, hi z: the ray's near and far ones
  // are loaded directly (per-ray offsets), no selects
  const float4* p = reinterpret_cast<const float4*>(node);
  const float4 nx = __ldg(p + r.sx), fx = __ldg(p + 1 - r.sx);
  const float4 ny = __ldg(p + 2 + r.sy), fy = __ldg(p + 3 - r.sy);
  const float4 nz = __ldg(p + 4 + r.sz), fz = __ldg(p + 5 - r.sz);
  int4 ch = __ldg(reinterpret_cast<const int4*>(p + 6));
  *child = ch;
  float nxa[4] = {nx.x, nx.y, nx.z, nx.w}, fxa[4] = {fx.x, fx.y, fx.z, fx.w};
  float nya[4] = {ny.x, ny.y, ny.z, ny.w}, fya[4] = {fy.x, fy.y, fy.z, fy.w};
  float nza[4] = {nz.x, nz.y, nz.z, nz.w}, fza[4] = {fz.x, fz.y, fz.z, fz.w};
  unsigned mask = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float t0 = fmaxf(fmaxf(__fmul_rn(__fsub_rn(nxa[i], r.ox), r.ix), __fmul_rn(__fsub_rn(nya[i], r.oy), r.iy)),
                     __fmul_rn(__fsub_rn(nza[i], r.oz), r.iz));
    float t1 = fminf(fminf(__fmul_rn(__fsub_rn(fxa[i], r.ox), r.ix), __fmul_rn(__fsub_rn(fya[i], r.oy), r.iy)),
                     __fmul_rn(__fsub_rn(fza[i], r.oz), r.iz));
    t0 = t0 - fabsf(t0) * kWiden;
    t1 = t1 + fabsf(t1) * kWiden;
    tn[i] = t0;
    if (t0 <= t1 && t0 <= bound && t1 >= r.tmin) mask |= 1u << i;
  }
  return mask;
}

// slab4 on a 64-byte node: decode the near and far planes of the four
// children (bytes on the node's per-axis grid) and run the same widened
// test; empty slots are masked by their child ref.
__device__ __forceinline__ unsigned slab4q(const QNode* __restrict__ node, const RayPre& r, float bound,
                                           float tn[4], int4* child) {
  const float4* p = reinterpret_cast<const float4*>(node);
  const float4 w0 = __ldg(p);
  const uint4 w1 = __ldg(reinterpret_cast<const uint4*>(p + 1));
  const uint4 w2 = __ldg(reinterpret_cast<const uint4*>(p + 2));
  const int4 ch = __ldg(reinterpret_cast<const int4*>(p + 3));
  *child = ch;
  const int ex = __float_as_int(w0.w);
  const float sx = qscale((ex & 255) - 128), sy = qscale(((ex >> 8) & 255) - 128), sz = qscale(((ex >> 16) & 255) - 128);
  const unsigned nxw = r.sx ? w1.y : w1.x, fxw = r.sx ? w1.x : w1.y;
  const unsigned nyw = r.sy ? w1.w : w1.z, fyw = r.sy ? w1.z : w1.w;
  const unsigned nzw = r.sz ? w2.y : w2.x, fzw = r.sz ? w2.x : w2.y;
  const int cha[4] = {ch.x, ch.y, ch.z, ch.w};
  unsigned mask = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const unsigned sel = 0x7540u + i;  // byte i of the word below 0x4B0000 (see qplane)
    const float nx = __fmaf_rn(__int_as_float(__byte_perm(nxw, 0x4B000000u, sel)) - 8388608.f, sx, w0.x);
    const float fx = __fmaf_rn(__int_as_float(__byte_perm(fxw, 0x4B000000u, sel)) - 8388608.f, sx, w0.x);
    const float ny = __fmaf_rn(__int_as_float(__byte_perm(nyw, 0x4B000000u, sel)) - 8388608.f, sy, w0.y);
    const float fy = __fmaf_rn(__int_as_float(__byte_perm(fyw, 0x4B000000u, sel)) - 8388608.f, sy, w0.y);
    const float nz = __fmaf_rn(__int_as_float(__byte_perm(nzw, 0x4B000000u, sel)) - 8388608.f, sz, w0.z);
    const float fz = __fmaf_rn(__int_as_float(__byte_perm(fzw, 0x4B000000u, sel)) - 8388608.f, sz, w0.z);
    float t0 = fmaxf(fmaxf(__fmul_rn(__fsub_rn(nx, r.ox), r.ix), __fmul_rn(__fsub_rn(ny, r.oy), r.iy)),
                     __fmul_rn(__fsub_rn(nz, r.oz), r.iz));
    float t1 = fminf(fminf(__fmul_rn(__fsub_rn(fx, r.ox), r.ix), __fmul_rn(__fsub_rn(fy, r.oy), r.iy)),
                     __fmul_rn(__fsub_rn(fz, r.oz), r.iz));
    t0 = t0 - fabsf(t0) * kWiden;
    t1 = t1 + fabsf(t1) * kWiden;
    tn[i] = t0;
    if (cha[i] != INT_MIN && t0 <= t1 && t0 <= bound && t1 >= r.tmin) mask |= 1u << i;
  }
  return mask;
}

// slab4 on an 8-wide node: the same widened test for its 8 children (two
// halves of four); empty slots have an empty box and never pass.
__device__ __forceinline__ unsigned slab8(const WNode8* __restrict__ node, const RayPre& r, float bound,
                                          float tn[8], int ch[8]) {
  const float4* p = reinterpret_cast<const float4*>(node);
  unsigned mask = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float4 nx = __ldg(p + 2 * r.sx + h), fx = __ldg(p + 2 - 2 * r.sx + h);
    const float4 ny = __ldg(p + 4 + 2 * r.sy + h), fy = __ldg(p + 6 - 2 * r.sy + h);
    const float4 nz = __ldg(p + 8 + 2 * r.sz + h), fz = __ldg(p + 10 - 2 * r.sz + h);
    const int4 c = __ldg(reinterpret_cast<const int4*>(p + 12 + h));
    ch[4 * h] = c.x;
    ch[4 * h + 1] = c.y;
    ch[4 * h + 2] = c.z;
    ch[4 * h + 3] = c.w;
    const float nxa[4] = {nx.x, nx.y, nx.z, nx.w}, fxa[4] = {fx.x, fx.y, fx.z, fx.w};
    const float nya[4] = {ny.x, ny.y, ny.z, ny.w}, fya[4] = {fy.x, fy.y, fy.z, fy.w};
    const float nza[4] = {nz.x, nz.y, nz.z, nz.w}, fza[4] = {fz.x, fz.y, fz.z, fz.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float t0 = fmaxf(fmaxf(__fmul_rn(__fsub_rn(nxa[i], r.ox), r.ix), __fmul_rn(__fsub_rn(nya[i], r.oy), r.iy)),
                       __fmul_rn(__fsub_rn(nza[i], r.oz), r.iz));
      float t1 = fminf(fminf(__fmul_rn(__fsub_rn(fxa[i], r.ox), r.ix), __fmul_rn(__fsub_rn(fya[i], r.oy), r.iy)),
                       __fmul_rn(__fsub_rn(fza[i], r.oz), r.iz));
      t0 = t0 - fabsf(t0) * kWiden;
      t1 = t1 + fabsf(t1) * kWiden;
      tn[4 * h + i] = t0;
      if (t0 <= t1 && t0 <= bound && t1 >= r.tmin) mask |= 1u << (4 * h + i);
    }
  }
  return mask;
}

// The same conservative slab test for one box (lo, hi) of a binary node.
__device__ __forceinline__ bool slab1(float4 lo, float4 hi, const RayPre& r, float bound) {
  const float nx = r.ix >= 0.f ? lo.x : hi.x, fx = r.ix >= 0.f ? hi.x : lo.x;
  const float ny = r.iy >= 0.f ? lo.y : hi.y, fy = r.iy >= 0.f ? hi.y : lo.y;
  const float nz = r.iz >= 0.f ? lo.z : hi.z, fz = r.iz >= 0.f ? hi.z : lo.z;
  float t0 = fmaxf(fmaxf(__fmul_rn(__fsub_rn(nx, r.ox), r.ix), __fmul_rn(__fsub_rn(ny, r.oy), r.iy)),
                   __fmul_rn(__fsub_rn(nz, r.oz), r.iz));
  float t1 = fminf(fminf(__fmul_rn(__fsub_rn(fx, r.ox), r.ix), __fmul_rn(__fsub_rn(fy, r.oy), r.iy)),
                   __fmul_rn(__fsub_rn(fz, r.oz), r.iz));
  t0 = t0 - fabsf(t0) * kWiden;
  t1 = t1 + fabsf(t1) * kWiden;
  return t0 <= t1 && t0 <= bound && t1 >= r.tmin;
}

__device__ __forceinline__ void cswap(float& ta, int& ra, float& tb, int& rb) {
  if (tb < ta) {
    float t = ta;
    ta = tb;
    tb = t;
    int x = ra;
    ra = rb;
    rb = x;
  }
}

__device__ __forceinline__ int enqueue_flag(int* counter, int* queue, int qcap, int i) {
  unsigned m = __activemask();
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(m, base, leader);
  int s = base + __popc(m & ((1u << lane) - 1u));
  if (s < qcap) {
    queue[s] = i;
    return s;
  }
  return -1;
}

struct TraceArgs {
  const WNode* wide;
  const WNode8* wide8;   // 8-wide nodes (walk with kW = 8)
  const int* wide_root;  // device word: index of the root traversal node
  const Node2* node2;
  const QNode* qwide;    // 64-byte nodes (walk with kQuant)
  const int2* link2;     // (parent, epoch) of every binary node
  const int* root_ref;   // device word: binary root (leaf ref if the root is a leaf)
  int n_tri;             // binary node ids are < n_tri - 1
  const float4* tris;
  const rt_ray* rays;
  int n;
  const int* n_dev;  // nullable: the number of rays lives on the device (<= n)
  rt_hit* hits;
  uint8_t* occl;
  const int32_t* skip;
  uint32_t* stats;
  int* counter;
  int* queue;
  int* cand;  // per queue slot: count (-1 = walk the whole tree) + kCand leaf positions
  int qcap;
};

// The float32 walk of ray i (the whole of Fig. 4 for one ray): results,
// statistics and the flag for the float64 pass.
template <bool kAny, bool kStats, int kSD, bool kQuant, int kW>
__device__ __forceinline__ void walk_one(const TraceArgs& A, const int i, const rt_ray* __restrict__ rays,
                                         rt_hit* __restrict__ hits, uint8_t* __restrict__ occl,
                                         const int32_t* __restrict__ skip_ids) {
  const float4* r4 = reinterpret_cast<const float4*>(rays) + 2 * (size_t)i;
  const RayPre r = setup_ray(__ldg(r4), __ldg(r4 + 1));
  const int skip = skip_ids ? __ldg(skip_ids + i) : -1;
  float t1 = INFINITY, t2 = INFINITY, e1 = 0.f, e2 = 0.f, bu = 0.f, bv = 0.f;
  int id1 = -1, pos1 = -1;
  bool flag = false, done = false;
  uint32_t n_nodes = 0, n_tris = 0;
  float bound = r.tmax;
  int2 st[kSD];  // (ref, entry distance bits) of the boxes still to visit
  int sp = 0;
  // Triangles whose float64 answer could beat the float32 one: uncertain
  // ones and every certain hit near the interval, with a lower bound on t.
  // If the ray is flagged, the float64 pass evaluates exactly these.
  int cpos[kCand];
  float clo[kCand];
  int nc = 0;
  bool walk_all = false;
  auto remember = [&](int pos, float lo) {
    if (nc == kCand) {  // make room: drop entries already beyond the cull bound
      int w = 0;
      for (int q = 0; q < kCand; ++q)
        if (clo[q] <= bound) {
          cpos[w] = cpos[q];
          clo[w] = clo[q];
          ++w;
        }
      nc = w;
    }
    if (nc < kCand) {
      cpos[nc] = pos;
      clo[nc] = lo;
      ++nc;
    } else {
      walk_all = true;
    }
  };
  // the node being visited stays in registers (cur); only the other
  // children hit by the ray go to the stack, nearest popped first
  int cur = r.valid ? __ldg(A.wide_root) : INT_MIN;
  float cur_t = -INFINITY;
  while (!done) {
    if (cur == INT_MIN) {
      if (sp == 0) break;
      --sp;
      cur = st[sp].x;
      cur_t = __int_as_float(st[sp].y);
    }
    const int ref = cur;
    cur = INT_MIN;
    if (cur_t > bound) continue;
    if (ref >= 0) {
      if (kStats) ++n_nodes;
      if (kW == 8) {
        float tn[8];
        int ch[8];
        const unsigned m = slab8(A.wide8 + ref, r, bound, tn, ch);
        const int cnt = __popc(m);
        if (cnt == 0) continue;
        if (sp + cnt - 1 > kSD) {  // cannot hold the children: leave it to the float64 pass
          flag = true;
          walk_all = true;
          break;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (!((m >> q) & 1u)) tn[q] = INFINITY;
        // sort the 8 (t, ref) pairs ascending (19 compare-exchanges)
        cswap(tn[0], ch[0], tn[2], ch[2]);
        cswap(tn[1], ch[1], tn[3], ch[3]);
        cswap(tn[4], ch[4], tn[6], ch[6]);
        cswap(tn[5], ch[5], tn[7], ch[7]);
        cswap(tn[0], ch[0], tn[4], ch[4]);
        cswap(tn[1], ch[1], tn[5], ch[5]);
        cswap(tn[2], ch[2], tn[6], ch[6]);
        cswap(tn[3], ch[3], tn[7], ch[7]);
        cswap(tn[0], ch[0], tn[1], ch[1]);
        cswap(tn[2], ch[2], tn[3], ch[3]);
        cswap(tn[4], ch[4], tn[5], ch[5]);
        cswap(tn[6], ch[6], tn[7], ch[7]);
        cswap(tn[2], ch[2], tn[4], ch[4]);
        cswap(tn[3], ch[3], tn[5], ch[5]);
        cswap(tn[1], ch[1], tn[4], ch[4]);
        cswap(tn[3], ch[3], tn[6], ch[6]);
        cswap(tn[1], ch[1], tn[2], ch[2]);
        cswap(tn[3], ch[3], tn[4], ch[4]);
        cswap(tn[5], ch[5], tn[6], ch[6]);
        // push farthest first so the nearest stacked one is popped next
#pragma unroll
        for (int q = 7; q >= 1; --q)
          if (q < cnt) st[sp++] = make_int2(ch[q], __float_as_int(tn[q]));
        cur = ch[0];
        cur_t = tn[0];
        continue;
      }
      float tn[4];
      int4 ch;
      unsigned m = kQuant ? slab4q(A.qwide + ref, r, bound, tn, &ch) : slab4(A.wide + ref, r, bound, tn, &ch);
      float ta = (m & 1u) ? tn[0] : INFINITY, tb = (m & 2u) ? tn[1] : INFINITY;
      float tc = (m & 4u) ? tn[2] : INFINITY, td = (m & 8u) ? tn[3] : INFINITY;
      int ra = ch.x, rb = ch.y, rc = ch.z, rd = ch.w;
      // sort 4 (t, ref) pairs ascending
      cswap(ta, ra, tb, rb);
      cswap(tc, rc, td, rd);
      cswap(ta, ra, tc, rc);
      cswap(tb, rb, td, rd);
      cswap(tb, rb, tc, rc);
      int cnt = __popc(m);
      if (cnt == 0) continue;
      if (sp + cnt - 1 > kSD) {  // cannot hold the children: leave it to the float64 pass
        flag = true;
        walk_all = true;
        break;
      }
      // push farthest first so the nearest stacked one is popped next
      if (cnt > 3) st[sp++] = make_int2(rd, __float_as_int(td));
      if (cnt > 2) st[sp++] = make_int2(rc, __float_as_int(tc));
      if (cnt > 1) st[sp++] = make_int2(rb, __float_as_int(tb));
      cur = ra;
      cur_t = ta;
      continue;
    }
    // leaf
    const int first = leaf_first(ref), count = leaf_count(ref);
    for (int k = 0; k < count; ++k) {
      const float4* tp = A.tris + 3 * (size_t)(first + k);
      float4 va = __ldg(tp), vb = __ldg(tp + 1), vc = __ldg(tp + 2);
      const int id = __float_as_int(va.w);
      if (id == skip) continue;
      if (kStats) ++n_tris;
      TriRes h = tri_test(r, va, vb, vc);
      if (h.cls == 0) continue;
      if (h.cls == 2) {
        if (h.thi >= r.tmin && h.tlo <= bound) {
          flag = true;
          remember(first + k, h.tlo);
        }
        continue;
      }
      // certain hit: near an end of the interval the float64 rule decides
      const bool near_end = fabsf(h.t - r.tmax) <= h.err + kTieRel * fabsf(r.tmax) ||
                            fabsf(h.t - r.tmin) <= h.err + kTieRel * fabsf(h.t);
      if (near_end) flag = true;
      if (near_end || (h.t > r.tmin && h.t < r.tmax)) remember(first + k, h.t - h.err);
      if (!(h.t > r.tmin && h.t < r.tmax)) continue;
      if (kAny) {
        if (!(fabsf(h.t - r.tmax) <= h.err + kTieRel * fabsf(r.tmax) ||
              fabsf(h.t - r.tmin) <= h.err + kTieRel * fabsf(h.t))) {
          done = true;
          id1 = id;
          break;
        }
        continue;
      }
      if (h.t < t1 || (h.t == t1 && id < id1)) {
        t2 = t1;
        e2 = e1;
        t1 = h.t;
        e1 = h.err;
        id1 = id;
        pos1 = first + k;
        bu = h.u;
        bv = h.v;
      } else if (h.t < t2) {
        t2 = h.t;
        e2 = h.err;
      }
      bound = fminf(r.tmax, t1 + kTieRel * t1 + e1);
    }
  }
  if (kAny) {
    occl[i] = done ? 1 : 0;
    if (done) flag = false;
  } else {
    if (t2 < INFINITY && t2 <= t1 + kTieRel * t1 + e1 + e2) flag = true;
    if (id1 >= 0 && e1 > 0.25f * (kTieRel * t1 + 1e-6f)) {
      // the float32 distance is not certified inside the tolerance: recompute it
      const float4* tp = A.tris + 3 * (size_t)pos1;
      const float4 rb4 = __ldg(r4 + 1);
      t1 = refine_t(r, rb4.x, rb4.y, rb4.z, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2));
    }
    float4 out = id1 >= 0 ? make_float4(t1, __int_as_float(id1), bu, bv)
                          : make_float4(INFINITY, __int_as_float(-1), 0.f, 0.f);
    reinterpret_cast<float4*>(hits)[i] = out;
  }
  if (kStats && A.stats) {
    A.stats[2 * (size_t)i] = n_nodes;
    A.stats[2 * (size_t)i + 1] = n_tris;
  }
  if (flag) {
    const int slot = enqueue_flag(A.counter, A.queue, A.qcap, i);
    if (slot >= 0) {
      int* c = A.cand + (size_t)slot * (kCand + 1);
      int w = 0;
      if (!walk_all)
        for (int q = 0; q < nc; ++q)
          if (clo[q] <= bound) c[1 + w++] = cpos[q];
      c[0] = walk_all ? -1 : w;
    }
  }
}

template <bool kAny, bool kStats, int kTile, int kSD, bool kQuant, int kW = 4>
__global__ void __launch_bounds__(kTile) k_trace(TraceArgs A) {
  const int i = blockIdx.x * kTile + threadIdx.x;
  if (i >= A.n || (A.n_dev && i >= *A.n_dev)) return;
  walk_one<kAny, kStats, kSD, kQuant, kW>(A, i, A.rays, A.hits, A.occl, A.skip);
}

// ---------------------------------------------------------------- float64
struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 dsub3(D3 a, D3 b) {
  return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)};
}
// (a.x*b.x + a.y*b.y) + a.z*b.z, rounded at every step
__device__ __forceinline__ double ddot(D3 a, D3 b) {
  double s = __dmul_rn(a.x, b.x);
  s = __dadd_rn(s, __dmul_rn(a.y, b.y));
  s = __dadd_rn(s, __dmul_rn(a.z, b.z));
  return s;
}
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
  return {__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)),
          __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
          __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x))};
}

// Moller-Trumbore, the reference hit rule (see file header).
__device__ bool mt64(D3 o, D3 d, D3 v0, D3 v1, D3 v2, double* t, double* u, double* v) {
  D3 e1 = dsub3(v1, v0), e2 = dsub3(v2, v0);
  D3 p = dcross(d, e2);
  double det = ddot(e1, p);
  double n1 = __dsqrt_rn(ddot(e1, e1)), n2 = __dsqrt_rn(ddot(e2, e2)), nd = __dsqrt_rn(ddot(d, d));
  double lim = __dmul_rn(1e-14, __dmul_rn(__dmul_rn(n1, n2), nd));
  if (fabs(det) <= lim) return false;
  double inv = __ddiv_rn(1.0, det);
  D3 s = dsub3(o, v0);
  double uu = __dmul_rn(ddot(s, p), inv);
  if (uu < 0.0 || uu > 1.0) return false;
  D3 q = dcross(s, e1);
  double vv = __dmul_rn(ddot(d, q), inv);
  if (vv < 0.0 || __dadd_rn(uu, vv) > 1.0) return false;
  *t = __dmul_rn(ddot(e2, q), inv);
  *u = uu;
  *v = vv;
  return true;
}

// Flagged rays with a candidate list: a group of G lanes each (G a power of
// two, the widest up to 32 that still gives every flagged ray its own group
// in this grid, so a handful of rays gets a warp each and a flood gets a
// thread each); lane q of a group tests candidates q, q + G, ... with the
// float64 rule and a reduction over the group keeps the nearest (lowest id on
// ties, the same minimum whatever G is).  Rays without a complete list: one
// thread each walks the tree.
// The float64 pass over every flagged ray, by threads tid of nthreads
// (nthreads a multiple of 32, whole warps).
template <bool kAny>
__device__ void retest_all(const TraceArgs& A, const int tid, const int nthreads, const rt_ray* __restrict__ rays,
                           rt_hit* __restrict__ hits, uint8_t* __restrict__ occl,
                           const int32_t* __restrict__ skip_ids) {
  const int nflag = min(*(volatile int*)A.counter, A.qcap);
  if (nflag <= 0) return;
  int lg = 5;
  while (lg > 0 && ((long long)nflag << lg) > nthreads) --lg;
  const int lane = threadIdx.x & 31, sub = lane & ((1 << lg) - 1);
  const int ngroups = nthreads >> lg;
  // jw: the first ray of this warp's groups; the loop is uniform over the warp
  for (int jw = (tid & ~31) >> lg; jw < nflag; jw += ngroups) {
    const int j = jw + (lane >> lg);
    const bool live = j < nflag;
    const int* cl = A.cand + (size_t)(live ? j : 0) * (kCand + 1);
    const int ncand = live ? cl[0] : -1;
    const int i = live ? A.queue[j] : 0;
    const float4* r4 = reinterpret_cast<const float4*>(rays) + 2 * (size_t)i;
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
    if (ncand > 0) {
      ra = r4[0];
      rb = r4[1];
    }
    const D3 o{ra.x, ra.y, ra.z}, d{rb.x, rb.y, rb.z};
    const double tmin = ra.w, tmax = rb.w;
    const int skip = (ncand > 0 && skip_ids) ? skip_ids[i] : -1;
    double bt = INFINITY, bu = 0.0, bv = 0.0;
    int bid = INT_MAX, bpos = -1;
    for (int q = sub; q < ncand; q += 1 << lg) {
      const int pos = cl[1 + q];
      const float4* tp = A.tris + 3 * (size_t)pos;
      const float4 va = tp[0], vb = tp[1], vc = tp[2];
      const int id = __float_as_int(va.w);
      double t, u, v;
      if (id != skip && mt64(o, d, D3{va.x, va.y, va.z}, D3{vb.x, vb.y, vb.z}, D3{vc.x, vc.y, vc.z}, &t, &u, &v) &&
          t > tmin && t < tmax && (t < bt || (t == bt && id < bid))) {
        bt = t;
        bid = id;
        bpos = pos;
        bu = u;
        bv = v;
      }
    }
    for (int off = (1 << lg) >> 1; off > 0; off >>= 1) {
      const double ot = __shfl_xor_sync(kFullMask, bt, off);
      const int oid = __shfl_xor_sync(kFullMask, bid, off);
      const int opos = __shfl_xor_sync(kFullMask, bpos, off);
      const double ou = __shfl_xor_sync(kFullMask, bu, off), ov = __shfl_xor_sync(kFullMask, bv, off);
      if (ot < bt || (ot == bt && oid < bid)) {
        bt = ot;
        bid = oid;
        bpos = opos;
        bu = ou;
        bv = ov;
      }
    }
    if (ncand < 0 || sub != 0) continue;  // a whole-tree walk is done below
    if (ncand == 0) {
      ra = r4[0];
      rb = r4[1];
    }
    const RayPre r = setup_ray(ra, rb);
    if (kAny) {
      occl[i] = bid != INT_MAX ? 1 : 0;
    } else {
      float4 out = make_float4(INFINITY, __int_as_float(-1), 0.f, 0.f);
      if (bid != INT_MAX) {
        out = make_float4((float)bt, __int_as_float(bid), (float)bu, (float)bv);
        // The record is a function of the ray and the winning triangle only:
        // where the float32 test certifies the winner, report exactly what
        // the float32 walk reports for it (so the result never depends on
        // whether this tree's walk flagged the ray).
        const float4* tp = A.tris + 3 * (size_t)bpos;
        const float4 va = tp[0], vb = tp[1], vc = tp[2];
        const TriRes h = tri_test(r, va, vb, vc);
        if (h.cls == 1 && h.t > r.tmin && h.t < r.tmax) {
          float t = h.t;
          if (h.err > 0.25f * (kTieRel * h.t + 1e-6f)) t = refine_t(r, rb.x, rb.y, rb.z, va, vb, vc);
          out = make_float4(t, __int_as_float(bid), h.u, h.v);
        }
      }
      reinterpret_cast<float4*>(hits)[i] = out;
    }
  }
  // rays without a complete candidate list: one thread each walks the tree
  for (int j = tid; j < nflag; j += nthreads) {
    const int i = A.queue[j];
    const float4* r4 = reinterpret_cast<const float4*>(rays) + 2 * (size_t)i;
    const float4 ra = r4[0], rb = r4[1];
    const RayPre r = setup_ray(ra, rb);
    const D3 o{ra.x, ra.y, ra.z}, d{rb.x, rb.y, rb.z};
    const double tmin = ra.w, tmax = rb.w;
    const int skip = skip_ids ? skip_ids[i] : -1;
    double bt = INFINITY, bu = 0.0, bv = 0.0;
    int bid = -1, bpos = -1;
    bool any = false;
    const int* cl = A.cand + (size_t)j * (kCand + 1);
    const int ncand = cl[0];
    if (ncand >= 0) continue;  // done by a warp above
    // Without a complete candidate list: a stackless walk of the binary tree
    // (parent links), so that any depth works.  Boxes use the same widened
    // float32 slab test as k_trace, culled at the float64 best distance
    // rounded up; triangles the float32 bound proves missed are skipped,
    // every other one goes through the float64 rule.
    auto test_leaf = [&](int ref) {
      const int first = leaf_first(ref), count = leaf_count(ref);
      for (int k = 0; k < count && !(kAny && any); ++k) {
        const float4* tp = A.tris + 3 * (size_t)(first + k);
        const float4 va = tp[0], vb = tp[1], vc = tp[2];
        const int id = __float_as_int(va.w);
        if (id == skip) continue;
        if (tri_test(r, va, vb, vc).cls == 0) continue;  // certain miss
        double t, u, v;
        if (mt64(o, d, D3{va.x, va.y, va.z}, D3{vb.x, vb.y, vb.z}, D3{vc.x, vc.y, vc.z}, &t, &u, &v) && t > tmin &&
            t < tmax) {
          any = true;
          if (t < bt || (t == bt && (bid < 0 || id < bid))) {
            bt = t;
            bid = id;
            bpos = first + k;
            bu = u;
            bv = v;
          }
        }
      }
    };
    if (r.valid) {
      const int root = *A.root_ref;
      if (root >= A.n_tri - 1) {
        // no usable tree: nothing to walk
      } else if (root < 0) {
        if (root != INT_MIN) test_leaf(root);
      } else {
        int node = root, s = 0;  // s: next child of `node` to try (2: done)
        for (long long guard = 0; guard < (1ll << 32); ++guard) {
          if (s < 2) {
            const Node2* nd = A.node2 + node;
            const float4 lo = s == 0 ? nd->a_lo : nd->b_lo, hi = s == 0 ? nd->a_hi : nd->b_hi;
            float bf = (float)fmin(bt, tmax);
            bf = bf + fabsf(bf) * 2e-6f;
            ++s;
            if (!slab1(lo, hi, r, bf)) continue;
            const int ref = __float_as_int(lo.w);
            if (ref >= 0) {
              if (ref < A.n_tri - 1) {  // a link the build never wrote is skipped
                node = ref;
                s = 0;
              }
              continue;
            }
            test_leaf(ref);
            if (kAny && any) break;
            continue;
          }
          if (node == root) break;
          const int p = A.link2[node].x;
          if (p < 0 || p >= A.n_tri - 1) break;
          s = __float_as_int(A.node2[p].a_lo.w) == node ? 1 : 2;
          node = p;
        }
      }
    }
    if (kAny) {
      occl[i] = any ? 1 : 0;
    } else {
      float4 out = make_float4(INFINITY, __int_as_float(-1), 0.f, 0.f);
      if (bid >= 0) {
        out = make_float4((float)bt, __int_as_float(bid), (float)bu, (float)bv);
        // The record is a function of the ray and the winning triangle only:
        // where the float32 test certifies the winner, report exactly what
        // the float32 walk reports for it (so the result never depends on
        // whether this tree's walk flagged the ray).
        const float4* tp = A.tris + 3 * (size_t)bpos;
        const float4 va = tp[0], vb = tp[1], vc = tp[2];
        const TriRes h = tri_test(r, va, vb, vc);
        if (h.cls == 1 && h.t > r.tmin && h.t < r.tmax) {
          float t = h.t;
          if (h.err > 0.25f * (kTieRel * h.t + 1e-6f)) t = refine_t(r, rb.x, rb.y, rb.z, va, vb, vc);
          out = make_float4(t, __int_as_float(bid), h.u, h.v);
        }
      }
      reinterpret_cast<float4*>(hits)[i] = out;
    }
  }
}

// Launched as a programmatic dependent of the walk: its CTAs are placed as
// the walk's last CTAs retire and wait here until the walk's results are
// visible.
template <bool kAny>
__global__ void __launch_bounds__(kRetestBlock) k_retest64(TraceArgs A) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  retest_all<kAny>(A, blockIdx.x * kRetestBlock + threadIdx.x, gridDim.x * kRetestBlock, A.rays, A.hits, A.occl,
                   A.skip);
}

// ---------------------------------------------------------------- one launch for a whole batch
// Every reflection order of a batch (Sec. III.B: trace, bounce, trace the
// bounced rays, until the order limit) and the visibility segments in one
// cooperative launch: the CTAs stay resident and step through the phases
// together, separated by grid barriers:
//   for each order k: walk (float32) -> barrier -> float64 pass of the flagged
//   rays -> barrier -> survivors per 32-ray chunk -> barrier -> offsets
//   (stable, in ray order) -> barrier -> bounce into order k + 1 -> barrier;
//   then the segments: walk (any hit) -> barrier -> float64 pass.
// The walk, the float64 pass and the bounce are the same device code as the
// separate kernels (rt_trace_closest, rt_reflect), so every order's rays,
// hits and parent indices are the same bits.  A barrier waits at most
// timeout_ns (global timer); when it runs out the status word is set and
// every CTA leaves.
struct PersistArgs {
  TraceArgs T;           // scene arrays and the float64 pass's scratch
  const float4* tri_in;  // input-order triangles (bounces)
  int max_order;
  int n0;
  rt_ray* rays[RT_BATCH_MAX_ORDER + 1];
  rt_hit* hits[RT_BATCH_MAX_ORDER + 1];
  int* skip[RT_BATCH_MAX_ORDER + 1];
  int* src[RT_BATCH_MAX_ORDER + 1];
  int* counts;       // counts[k]: rays of order k >= 1 (written here)
  int* chunk;        // per 32-ray chunk: survivors, then the chunk's first output position
  int* cta_total;    // per CTA: survivors of its chunks
  const rt_ray* seg;
  int n_seg;
  uint8_t* occl;
  unsigned* bar;     // [0] arrivals, [1] generation (zero before the launch)
  int* status;       // 0, or 1 when a barrier ran out of time
  int* take;         // [RT_BATCH_MAX_ORDER + 2]: rays handed out so far by each walk phase (orders,
                     // then the segments; zero before)
  long long timeout_ns;
  int receive;       // 1: carry each ray's delta (reception, Eq. 4) through the bounces
  float* delta[RT_BATCH_MAX_ORDER + 1];
};

constexpr int kPersistBlock = 128;
constexpr int kPersistMinBlocks = 8;  // 64 registers: the walk's own budget

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier (all CTAs resident: cooperative launch).  Returns false when
// the batch failed (a barrier ran out of time); the caller then leaves.
__device__ bool grid_sync(const PersistArgs& P) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* arrive = P.bar;
    volatile unsigned* gen = P.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(arrive, 1u) == gridDim.x - 1) {
      atomicExch(arrive, 0u);
      __threadfence();
      atomicAdd(P.bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (*(volatile int*)P.status != 0) {
          good = 0;
          break;
        }
        if (global_ns() - t0 > (unsigned long long)P.timeout_ns) {
          atomicCAS(P.status, 0, 1);
          good = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok = good && *(volatile int*)P.status == 0;
  }
  __syncthreads();
  return ok;
}

// A walk phase: every warp takes batches of 32 rays (a ray per lane) from
// the phase's device counter until none is left, so the CTAs that drew cheap
// rays take more and the phase ends with the last rays.  (Batches of 64,
// two walks per lane one after the other, made every warp wait for its
// slowest lane twice per claim.)
template <bool kAny, int kW>
__device__ __forceinline__ void walk_phase(const TraceArgs& A, int* take, int n, const rt_ray* rays, rt_hit* hits,
                                           uint8_t* occl, const int* skip) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int b = 0;
    if (lane == 0) b = atomicAdd(take, 32);
    b = __shfl_sync(kFullMask, b, 0);
    if (b >= n) break;
    if (b + lane < n) walk_one<kAny, false, kStack, false, kW>(A, b + lane, rays, hits, occl, skip);
  }
}

__device__ __forceinline__ bool bounces(const rt_hit* hits, const rt_ray* rays, int i) {
  const float4 h = reinterpret_cast<const float4*>(hits)[i];
  const float tmax = reinterpret_cast<const float4*>(rays)[2 * (size_t)i + 1].w;
  return __float_as_int(h.y) >= 0 && tmax - h.x > 0.f;
}

template <int kW>
__global__ void __launch_bounds__(kPersistBlock, kPersistMinBlocks) k_batch(const __grid_constant__ PersistArgs P) {
  __shared__ int red[kPersistBlock / 32];
  __shared__ int carry;
  const int nth = gridDim.x * kPersistBlock;
  const int tid = blockIdx.x * kPersistBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kPersistBlock / 32;
  const TraceArgs& A = P.T;  // scene arrays (stats, occl, n_dev unused here)
  for (int k = 0;; ++k) {
    const int n = k == 0 ? P.n0 : *(volatile int*)(P.counts + k);
    const rt_ray* rays = P.rays[k];
    rt_hit* hits = P.hits[k];
    const int* skip = k ? P.skip[k] : nullptr;
    walk_phase<false, kW>(A, P.take + k, n, rays, hits, nullptr, skip);
    if (!grid_sync(P)) return;
    retest_all<false>(A, tid, nth, rays, hits, nullptr, skip);
    if (!grid_sync(P)) return;
    if (k == P.max_order) break;
    // survivors of the bounce per 32-ray chunk; CTA b owns a contiguous run of chunks
    if (tid == 0) *A.counter = 0;  // the next order's flags (this order's float64 pass is done)
    const int nch = (n + 31) / 32, per = (nch + (int)gridDim.x - 1) / (int)gridDim.x;
    const int c0 = min(nch, (int)blockIdx.x * per), c1 = min(nch, c0 + per);
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c = c0 + warp; c < c1; c += kWarps) {
      const int i = c * 32 + lane;
      const unsigned m = __ballot_sync(kFullMask, i < n && bounces(hits, rays, i));
      if (lane == 0) {
        P.chunk[c] = __popc(m);
        atomicAdd(&carry, __popc(m));
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) P.cta_total[blockIdx.x] = carry;
    if (!grid_sync(P)) return;
    // first output position of every chunk: the survivors of the CTAs before
    // this one, then a scan over this CTA's chunks in order
    {
      int part = 0;
      for (int b = threadIdx.x; b < (int)blockIdx.x; b += kPersistBlock) part += P.cta_total[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFullMask, part, o);
      if (lane == 0) red[warp] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kWarps; ++w) t += red[w];
        carry = t;
      }
      __syncthreads();
      for (int t0 = c0; t0 < c1; t0 += kPersistBlock) {
        const int c = t0 + threadIdx.x;
        const int v = c < c1 ? P.chunk[c] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFullMask, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) red[warp] = x;
        __syncthreads();
        int off = carry, tot = 0;
        for (int w = 0; w < kWarps; ++w) {
          if (w < warp) off += red[w];
          tot += red[w];
        }
        if (c < c1) P.chunk[c] = off + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
      }
      if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) P.counts[k + 1] = carry;
    }
    if (!grid_sync(P)) return;
    // the bounce: every surviving ray of the chunk at its place in order k + 1
    for (int c = c0 + warp; c < c1; c += kWarps) {
      const int i = c * 32 + lane;
      const bool keep = i < n && bounces(hits, rays, i);
      const unsigned m = __ballot_sync(kFullMask, keep);
      if (!keep) continue;
      const int pos = P.chunk[c] + __popc(m & ((1u << lane) - 1u));
      const float4* r4 = reinterpret_cast<const float4*>(rays) + 2 * (size_t)i;
      const float4 h = reinterpret_cast<const float4*>(hits)[i];
      const int id = __float_as_int(h.y);
      float4 o0, o1;
      reflect_ray(r4[0], r4[1], h.x, P.tri_in[3 * (size_t)id], P.tri_in[3 * (size_t)id + 1],
                  P.tri_in[3 * (size_t)id + 2], &o0, &o1);
      float4* out = reinterpret_cast<float4*>(P.rays[k + 1]) + 2 * (size_t)pos;
      out[0] = o0;
      out[1] = o1;
      P.skip[k + 1][pos] = id;
      P.src[k + 1][pos] = i;
      if (P.receive) P.delta[k + 1][pos] = P.delta[k][i];
    }
    if (!grid_sync(P)) return;
  }
  if (P.n_seg > 0) {
    if (tid == 0) *A.counter = 0;
    if (!grid_sync(P)) return;
    walk_phase<true, kW>(A, P.take + RT_BATCH_MAX_ORDER + 1, P.n_seg, P.seg, nullptr, P.occl, nullptr);
    if (!grid_sync(P)) return;
    retest_all<true>(A, tid, nth, P.seg, nullptr, P.occl, nullptr);
  }
}

int sm_count_t() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

cudaError_t launch_trace(rt_scene_s* s, const rt_ray* rays, int64_t n, rt_hit* hits, uint8_t* occl,
                         const rt_trace_params* tp, TraceScratch& scr, cudaStream_t st) {
  return launch_trace_dev(s, rays, n, nullptr, hits, occl, tp, scr, st);
}

namespace {

template <bool kAny, bool kStats, int kTile, int kSD, bool kQuant, int kW = 4>
void walk(const TraceArgs& A, int64_t n, cudaStream_t st) {
  k_trace<kAny, kStats, kTile, kSD, kQuant, kW><<<(int)((n + kTile - 1) / kTile), kTile, 0, st>>>(A);
}

// The tuned walks: node width 4 / 8 x ray tile 64 / 128 / 256 x stack depth
// 16 / 32 / 64.
template <bool kAny, int kTile, int kW>
void walk_stack(const TraceArgs& A, int64_t n, int stack, cudaStream_t st) {
  if (stack == 16)
    walk<kAny, false, kTile, 16, false, kW>(A, n, st);
  else if (stack == 32)
    walk<kAny, false, kTile, 32, false, kW>(A, n, st);
  else
    walk<kAny, false, kTile, 64, false, kW>(A, n, st);
}
template <bool kAny, int kW>
void walk_tile(const TraceArgs& A, int64_t n, int tile, int stack, cudaStream_t st) {
  if (tile == 64)
    walk_stack<kAny, 64, kW>(A, n, stack, st);
  else if (tile == 256)
    walk_stack<kAny, 256, kW>(A, n, stack, st);
  else
    walk_stack<kAny, 128, kW>(A, n, stack, st);
}
template <bool kAny>
void walk_tuned(const TraceArgs& A, int64_t n, int width, int tile, int stack, cudaStream_t st) {
  if (width == 8)
    walk_tile<kAny, 8>(A, n, tile, stack, st);
  else
    walk_tile<kAny, 4>(A, n, tile, stack, st);
}

}  // namespace

cudaError_t launch_trace_dev(rt_scene_s* s, const rt_ray* rays, int64_t n, const int* n_dev, rt_hit* hits,
                             uint8_t* occl, const rt_trace_params* tp, TraceScratch& scr, cudaStream_t st) {
  cudaError_t e;
  int n_launched = 0;
  const bool quant = tp && (tp->flags & RT_QUANTIZED_NODES);
  if (quant && !s->q_built) return cudaErrorInvalidValue;  // no 64-byte nodes for this tree
  const int width = s->params.width == 8 ? 8 : 4;          // the traversal nodes the last build wrote
  if ((e = cudaMemsetAsync(scr.counter, 0, 2 * sizeof(int), st))) return e;
  if (n > 0) {
    TraceArgs A;
    A.wide = s->wide;
    A.wide8 = s->wide8;
    A.qwide = s->qwide;
    A.wide_root = &s->ctl->wide_root;
    A.node2 = s->node2;
    A.link2 = s->link2;
    A.root_ref = &s->ctl->root_ref;
    A.n_tri = (int)s->n_built;
    A.tris = s->tri_leaf;
    A.rays = rays;
    A.n = (int)n;
    A.n_dev = n_dev;
    A.hits = hits;
    A.occl = occl;
    A.skip = tp ? tp->skip_tri_dev : nullptr;
    const bool stats = tp && (tp->flags & RT_COUNT_STATS) && tp->stats_dev;
    A.stats = stats ? tp->stats_dev : nullptr;
    A.counter = scr.counter;
    A.queue = scr.queue;
    A.cand = scr.cand;
    A.qcap = (int)scr.cap;
    // ray tile (rays per CTA) and stack depth; the counting walk and the
    // 64-byte node walk use the defaults
    const int tile = (tp && !stats && !quant && (tp->block == 64 || tp->block == 256)) ? tp->block : kTraceBlock;
    const int stack = (tp && !stats && !quant && (tp->stack == 16 || tp->stack == 32)) ? tp->stack : kStack;
    if (quant) {
      if (occl)
        stats ? walk<true, true, kTraceBlock, kStack, true>(A, n, st)
              : walk<true, false, kTraceBlock, kStack, true>(A, n, st);
      else
        stats ? walk<false, true, kTraceBlock, kStack, true>(A, n, st)
              : walk<false, false, kTraceBlock, kStack, true>(A, n, st);
    } else if (stats) {
      if (width == 8)
        occl ? walk<true, true, kTraceBlock, kStack, false, 8>(A, n, st)
             : walk<false, true, kTraceBlock, kStack, false, 8>(A, n, st);
      else
        occl ? walk<true, true, kTraceBlock, kStack, false>(A, n, st)
             : walk<false, true, kTraceBlock, kStack, false>(A, n, st);
    } else {
      occl ? walk_tuned<true>(A, n, width, tile, stack, st) : walk_tuned<false>(A, n, width, tile, stack, st);
    }
    ++n_launched;
    if (!(tp && (tp->flags & RT_NO_FP64_RETEST))) {
      int g = (int)((n + kRetestBlock - 1) / kRetestBlock);
      int gmax = sm_count_t() * 4;
      g = g < gmax ? g : gmax;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)g);
      cfg.blockDim = dim3(kRetestBlock);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if ((e = occl ? cudaLaunchKernelEx(&cfg, k_retest64<true>, A) : cudaLaunchKernelEx(&cfg, k_retest64<false>, A)))
        return e;
      ++n_launched;
    }
  }
  if (tp && tp->n_flagged_dev) {
    if ((e = cudaMemcpyAsync(tp->n_flagged_dev, scr.counter, sizeof(int), cudaMemcpyDeviceToDevice, st)))
      return e;
  }
  count_launches(n_launched);
  return cudaGetLastError();
}

cudaError_t launch_batch_persistent(rt_scene_s* s, const BatchLaunch& b, cudaStream_t st) {
  PersistArgs P;
  TraceArgs& A = P.T;
  A.wide = s->wide;
  A.wide8 = s->wide8;
  A.qwide = s->qwide;
  A.wide_root = &s->ctl->wide_root;
  A.node2 = s->node2;
  A.link2 = s->link2;
  A.root_ref = &s->ctl->root_ref;
  A.n_tri = (int)s->n_built;
  A.tris = s->tri_leaf;
  A.counter = b.scr->counter;
  A.queue = b.scr->queue;
  A.cand = b.scr->cand;
  A.qcap = (int)b.scr->cap;
  A.n_dev = nullptr;
  A.stats = nullptr;
  P.tri_in = s->tri_in;
  P.max_order = b.max_order;
  P.n0 = (int)b.n0;
  for (int k = 0; k <= RT_BATCH_MAX_ORDER; ++k) {
    P.rays[k] = b.rays[k];
    P.hits[k] = b.hits[k];
    P.skip[k] = b.skip[k];
    P.src[k] = b.src[k];
  }
  P.counts = b.counts;
  P.chunk = b.chunk;
  P.cta_total = b.cta_total;
  P.seg = b.seg;
  P.n_seg = (int)b.n_seg;
  P.occl = b.occl;
  P.bar = b.bar;
  P.status = b.status;
  P.take = b.take;
  P.receive = b.receive;
  for (int k = 0; k <= RT_BATCH_MAX_ORDER; ++k) P.delta[k] = b.delta[k];
  P.timeout_ns = b.timeout_ns;
  cudaError_t e;
  // arrivals, generation, status and the phases' ray counters start from
  // zero; the flag counter too
  if ((e = cudaMemsetAsync(b.bar, 0, 4 * sizeof(unsigned), st))) return e;
  if ((e = cudaMemsetAsync(b.take, 0, (RT_BATCH_MAX_ORDER + 2) * sizeof(int), st))) return e;
  if ((e = cudaMemsetAsync(b.scr->counter, 0, 2 * sizeof(int), st))) return e;
  const bool w8 = s->params.width == 8;
  void (*k)(PersistArgs) = w8 ? k_batch<8> : k_batch<4>;
  static int per_sm[2] = {0, 0};
  int& ps = per_sm[w8 ? 1 : 0];
  if (!ps) {
    int nb = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kPersistBlock, 0))) return e;
    ps = nb;
  }
  if (ps < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int grid = std::min(ps * sm_count_t(), b.cta_cap);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPersistBlock);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if ((e = cudaLaunchKernelEx(&cfg, k, P))) return e;
  count_launches(1);
  return cudaSuccess;
}

int persistent_batch_ctas() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<4>, kPersistBlock, 0);
  int nb8 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb8, k_batch<8>, kPersistBlock, 0);
  return std::max(std::max(nb, nb8), 1) * sm_count_t();
}

}  // namespace rt
